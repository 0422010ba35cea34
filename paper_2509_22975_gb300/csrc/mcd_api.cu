// extern "C" entry points declared in include/mcd.h: argument checks, state
// handling and dispatch to the sampler, index, H*v and Lanczos code.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>

#include "mcd_internal.h"

namespace mcd {

int fail(mcd_ctx* c, int status, const std::string& msg) {
  if (c) c->err = msg;
  return status;
}

int cuda_fail(mcd_ctx* c, cudaError_t e, const char* where) {
  return fail(c, MCD_E_CUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

int device_sms() {
  constexpr int kDevs = 64;
  static std::atomic<int> cached[kDevs] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  if (dev < kDevs) {
    const int v = cached[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  if (dev < kDevs) cached[dev].store(v, std::memory_order_relaxed);
  return v;
}

}  // namespace mcd

using namespace mcd;

namespace {

const char* g_create_error = "";

bool has_device(mcd_ctx* c) { return c->device >= 0; }

int need_device(mcd_ctx* c) {
  if (!has_device(c)) return fail(c, MCD_E_NODEVICE, "host-only context (device = -1)");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return MCD_OK;
}

int need_basis(mcd_ctx* c) {
  if (!c->has_ham) return fail(c, MCD_E_STATE, "no Hamiltonian set");
  if (c->n_basis == 0) return fail(c, MCD_E_STATE, "no basis set");
  return MCD_OK;
}

int install_basis(mcd_ctx* c, std::vector<uint64_t>&& words) {
  c->gs_valid = false;
  c->basis = std::move(words);
  c->n_basis = int64_t(c->basis.size());
  c->basis_on_host = true;
  if (has_device(c)) {
    int st = need_device(c);
    if (st != MCD_OK) return st;
    st = build_index(c, c->basis.data(), c->n_basis, false);
    if (st != MCD_OK) {
      c->basis.clear();
      c->n_basis = 0;
      return st;
    }
  }
  return MCD_OK;
}

}  // namespace

namespace {

// f(i, ctx) for every instance, on a pool of host threads: each thread owns a
// non-blocking CUDA stream that it sets on the instance's context for the
// call (the context's stream is restored afterwards), so instances run
// concurrently on the GPU.  Returns the status of the first failing instance
// (lowest index; an error before a mere MCD_E_NOT_CONVERGED), its message in
// ctxs[0]'s last error.
template <typename F>
int run_instances(mcd_ctx* const* ctxs, int n, F f) {
  const int hw = int(std::thread::hardware_concurrency());
  const int nthreads = std::max(1, std::min(n, std::min(hw > 0 ? hw : 1, 16)));
  std::atomic<int> next{0};
  std::mutex mu;
  int err_idx = -1, err_st = MCD_OK;
  std::string err_msg;
  auto note = [&](int i, int st, const std::string& msg) {
    std::lock_guard<std::mutex> lock(mu);
    const bool soft = st == MCD_E_NOT_CONVERGED, was_soft = err_st == MCD_E_NOT_CONVERGED;
    if (err_idx < 0 || (was_soft && !soft) || (soft == was_soft && i < err_idx)) {
      err_idx = i;
      err_st = st;
      err_msg = msg;
    }
  };
  auto worker = [&]() {
    cudaSetDevice(ctxs[0]->device);
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      note(0, MCD_E_CUDA, std::string("batch stream: ") + cudaGetErrorString(e));
      return;
    }
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      mcd_ctx* c = ctxs[i];
      cudaStream_t old = c->stream;
      int st = mcd_set_stream(c, s);
      if (st == MCD_OK) st = f(i, c);
      const std::string msg = c->err;
      const int st2 = mcd_set_stream(c, old);   // waits for this instance's work
      if (st == MCD_OK) st = st2;
      if (st != MCD_OK) note(i, st, msg);
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  pool.reserve(nthreads);
  for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  if (err_idx >= 0) return fail(ctxs[0], err_st, "instance " + std::to_string(err_idx) + ": " + err_msg);
  return MCD_OK;
}

int check_instances(mcd_ctx* const* ctxs, int n, bool same_sites) {
  if (!ctxs || n < 1 || !ctxs[0]) return MCD_E_INVALID;
  for (int i = 0; i < n; ++i) {
    mcd_ctx* c = ctxs[i];
    if (!c) return fail(ctxs[0], MCD_E_INVALID, "batch: null context");
    if (c->device != ctxs[0]->device) return fail(ctxs[0], MCD_E_INVALID, "batch: contexts on different devices");
    if (same_sites && c->n != ctxs[0]->n) return fail(ctxs[0], MCD_E_INVALID, "batch: instances differ in sites");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(ctxs[0], MCD_E_INVALID, "batch: a context appears twice");
  }
  return MCD_OK;
}

}  // namespace

extern "C" {

int mcd_create(mcd_ctx** out, int device, void* cuda_stream) {
  if (!out) return MCD_E_INVALID;
  *out = nullptr;
  mcd_ctx* c = new (std::nothrow) mcd_ctx();
  if (!c) {
    g_create_error = "out of host memory";
    return MCD_E_OOM;
  }
  c->hp = new (std::nothrow) HamParams();
  if (!c->hp) {
    delete c;
    g_create_error = "out of host memory";
    return MCD_E_OOM;
  }
  std::memset(c->hp, 0, sizeof(HamParams));
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (device >= 0) {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device >= count) {
      g_create_error = e != cudaSuccess ? cudaGetErrorString(e) : "device ordinal out of range";
      delete c->hp;
      delete c;
      return e != cudaSuccess ? MCD_E_CUDA : MCD_E_INVALID;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) {
      g_create_error = cudaGetErrorString(e);
      delete c->hp;
      delete c;
      return MCD_E_CUDA;
    }
  } else if (device != -1) {
    g_create_error = "device must be >= 0 or -1 (host only)";
    delete c->hp;
    delete c;
    return MCD_E_INVALID;
  }
  *out = c;
  return MCD_OK;
}

int mcd_destroy(mcd_ctx* c) {
  if (!c) return MCD_OK;
  if (has_device(c)) {
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_index(c->idx, c->stream);
    free_lanczos(c->lw);
    if (c->d_eps) cudaFreeAsync(c->d_eps, c->stream);
    if (c->d_U) cudaFreeAsync(c->d_U, c->stream);
    if (c->d_pclass) cudaFreeAsync(c->d_pclass, c->stream);
    if (c->gs_psi) cudaFreeAsync(c->gs_psi, c->stream);
    cudaStreamSynchronize(c->stream);
    for (auto& ev : c->tune_ev)
      if (ev) cudaEventDestroy(ev);
    if (c->tm && !c->tm_borrowed) {
      if (c->tm->created)
        for (auto& ev : c->tm->ev) cudaEventDestroy(ev);
      delete c->tm;
    }
  }
  delete c->hp;
  delete c;
  return MCD_OK;
}

int mcd_set_stream(mcd_ctx* c, void* stream) {
  if (!c) return MCD_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (has_device(c) && s != c->stream) {
    // the context's buffers are allocated and freed in the order of its
    // stream: the old stream's work completes before the new one is used
    cudaSetDevice(c->device);
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronise the previous stream");
  }
  c->stream = s;
  return MCD_OK;
}

int mcd_set_option(mcd_ctx* c, int option, int64_t value) {
  if (!c) return MCD_E_INVALID;
  switch (option) {
    case MCD_OPT_HV_ALGO:
      if (value < 0 || value > 3) return fail(c, MCD_E_INVALID, "HV_ALGO must be 0, 1, 2 or 3");
      c->hv_algo = int(value);
      return MCD_OK;
    case MCD_OPT_KERNEL_TIMING:
      if (value && has_device(c)) {
        int st = need_device(c);
        if (st != MCD_OK) return st;
        if (!c->tm) c->tm = new (std::nothrow) Timing();
        if (!c->tm) return fail(c, MCD_E_OOM, "timing");
        if (!c->tm->created) {
          for (auto& ev : c->tm->ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
          }
          c->tm->created = true;
        }
      }
      c->timing = value ? 1 : 0;
      return MCD_OK;
    case MCD_OPT_HASH_ITEM:
      if (value < 64 || value > 4096 || (value & (value - 1)))
        return fail(c, MCD_E_INVALID, "HASH_ITEM must be a power of two in [64, 4096]");
      c->hash_item = int(value);
      return MCD_OK;
    case MCD_OPT_SAMPLER_DEVICE:
      if (value < 0 || value > 2) return fail(c, MCD_E_INVALID, "SAMPLER_DEVICE must be 0, 1 or 2");
      c->sampler_where = int(value);
      return MCD_OK;
    case MCD_OPT_KRYLOV_STORE:
      if (value < 0 || value > 1) return fail(c, MCD_E_INVALID, "KRYLOV_STORE must be 0 or 1");
      c->krylov_store = int(value);
      return MCD_OK;
    case MCD_OPT_HV_COLS:
      if (value < 0 || value > 2) return fail(c, MCD_E_INVALID, "HV_COLS must be 0, 1 or 2");
      c->hv_cols = int(value);
      return MCD_OK;
    case MCD_OPT_BATCH_MODE:
      if (value < 0 || value > 1) return fail(c, MCD_E_INVALID, "BATCH_MODE must be 0 or 1");
      c->batch_mode = int(value);
      return MCD_OK;
    case MCD_OPT_BATCH_SPLIT:
      if (value != 0 && value != 1 && value != 2 && value != 4)
        return fail(c, MCD_E_INVALID, "BATCH_SPLIT must be 0, 1, 2 or 4");
      c->batch_split = int(value);
      return MCD_OK;
    case MCD_OPT_APPLY_SYNC:
      if (value < 0 || value > 1) return fail(c, MCD_E_INVALID, "APPLY_SYNC must be 0 or 1");
      c->apply_sync = int(value);
      return MCD_OK;
    case MCD_OPT_WAIT_TEST:
      if (value < -1) return fail(c, MCD_E_INVALID, "WAIT_TEST must be -1 or an item index");
      c->wait_test_item = value;
      return MCD_OK;
    case MCD_OPT_HV_CACHE:
      if (value < 0 || value > 2) return fail(c, MCD_E_INVALID, "HV_CACHE must be 0, 1 or 2");
      c->hv_cache = int(value);
      if (value == 1 && has_device(c)) {   // release the records
        free_cache(c->idx.A, c->stream);
        free_cache(c->idx.B, c->stream);
      }
      return MCD_OK;
    case MCD_OPT_SAMPLER_THREADS:
      if (value < 0 || value > 1024) return fail(c, MCD_E_INVALID, "SAMPLER_THREADS out of range");
      c->sampler_threads = int(value);
      return MCD_OK;
    default:
      return fail(c, MCD_E_INVALID, "unknown option");
  }
}

const char* mcd_last_error(const mcd_ctx* c) { return c ? c->err.c_str() : g_create_error; }

const char* mcd_status_string(int s) {
  switch (s) {
    case MCD_OK: return "ok";
    case MCD_W_SHORT: return "sampler returned fewer states than asked";
    case MCD_E_INVALID: return "invalid argument";
    case MCD_E_SECTOR: return "state outside the sector";
    case MCD_E_OOM: return "out of memory";
    case MCD_E_CUDA: return "CUDA error";
    case MCD_E_NOT_CONVERGED: return "not converged";
    case MCD_E_BREAKDOWN: return "Lanczos breakdown";
    case MCD_E_TIMEOUT: return "timeout";
    case MCD_E_STATE: return "call out of order";
    case MCD_E_NODEVICE: return "no device in this context";
    default: return "unknown status";
  }
}

int mcd_set_hamiltonian(mcd_ctx* c, int n, const double* t, const double* eps, const double* U, int U_len,
                        int n_up, int n_dn) {
  if (!c) return MCD_E_INVALID;
  if (n < 1 || n > kMaxSites) return fail(c, MCD_E_INVALID, "n_sites must be in [1, 32]");
  if (!t || !U) return fail(c, MCD_E_INVALID, "t and U are required");
  if (U_len != 1 && U_len != n) return fail(c, MCD_E_INVALID, "U_len must be 1 or n_sites");
  if (n_up < 0 || n_dn < 0 || n_up > n || n_dn > n) return fail(c, MCD_E_INVALID, "bad N_up / N_dn");
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double v = t[size_t(i) * n + j];
      if (!std::isfinite(v)) return fail(c, MCD_E_INVALID, "non-finite t_ij");
      if (i != j && v != t[size_t(j) * n + i]) return fail(c, MCD_E_INVALID, "t must be symmetric");
    }
  std::vector<double> e(n, 0.0), u(n, 0.0);
  for (int i = 0; i < n; ++i) {
    e[i] = eps ? eps[i] : 0.0;
    u[i] = U[U_len == 1 ? 0 : i];
    if (!std::isfinite(e[i]) || !std::isfinite(u[i])) return fail(c, MCD_E_INVALID, "non-finite eps or U");
  }
  const bool sector_changed = !c->has_ham || n != c->n || n_up != c->n_up || n_dn != c->n_dn;
  c->n = n;
  c->n_up = n_up;
  c->n_dn = n_dn;
  c->t.assign(t, t + size_t(n) * n);
  c->eps = e;
  c->U = u;
  HamParams& hp = *c->hp;
  std::memset(&hp, 0, sizeof(HamParams));
  hp.n_sites = n;
  int nb = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double v = t[size_t(i) * n + j];
      if (v == 0.0) continue;
      Bond& b = hp.bonds[nb++];
      b.mask = (1u << i) | (1u << j);
      b.between = (j - i > 1) ? (((j >= 32 ? 0u : (1u << j)) - 1u) & ~((1u << (i + 1)) - 1u)) : 0u;
      b.t = v;
      b.t_hi = float(v);
      b.t_lo = float(v - double(b.t_hi));
    }
  hp.n_bonds = nb;
  // group bonds by amplitude (stable), so kernels can sum +-x per class and
  // multiply by t once
  {
    std::vector<double> vals;
    for (int b = 0; b < nb; ++b) {
      bool seen = false;
      for (double v : vals) seen |= (v == hp.bonds[b].t);
      if (!seen) vals.push_back(hp.bonds[b].t);
    }
    if (int(vals.size()) <= kMaxClasses) {
      std::vector<Bond> sorted;
      sorted.reserve(nb);
      hp.n_class = int(vals.size());
      for (int cidx = 0; cidx < hp.n_class; ++cidx) {
        for (int b = 0; b < nb; ++b)
          if (hp.bonds[b].t == vals[cidx]) sorted.push_back(hp.bonds[b]);
        hp.cls_end[cidx] = int(sorted.size());
        hp.cls_t[cidx] = vals[cidx];
        hp.cls_hi[cidx] = float(vals[cidx]);
        hp.cls_lo[cidx] = float(vals[cidx] - double(hp.cls_hi[cidx]));
      }
      for (int b = 0; b < nb; ++b) hp.bonds[b] = sorted[b];
    } else {
      hp.n_class = 0;
    }
  }
  // hop groups: bonds of equal amplitude and equal index distance j - i
  {
    hp.n_hg = 0;
    bool ok = true;
    for (int b = 0; b < nb && ok; ++b) {
      const int i = __builtin_ctz(hp.bonds[b].mask);
      const int j = 31 - __builtin_clz(hp.bonds[b].mask);
      int g = 0;
      while (g < hp.n_hg && !(hp.hg_t[g] == hp.bonds[b].t && hp.hg_shift[g] == j - i)) ++g;
      if (g == hp.n_hg) {
        if (g == kMaxHopGroups) { ok = false; break; }
        hp.hg_t[g] = hp.bonds[b].t;
        hp.hg_hi[g] = hp.bonds[b].t_hi;
        hp.hg_lo[g] = hp.bonds[b].t_lo;
        hp.hg_shift[g] = j - i;
        hp.hg_mask[g] = 0u;
        ++hp.n_hg;
      }
      hp.hg_mask[g] |= 1u << i;
    }
    if (!ok) hp.n_hg = 0;
  }
  bool uniform = true;
  for (int i = 1; i < n; ++i)
    if (e[i] != e[0] || u[i] != u[0]) uniform = false;
  hp.uniform = uniform ? 1 : 0;
  if (uniform) {
    for (int k = 0; k <= n; ++k) {
      const double d = e[0] * double(n_up + n_dn) + u[0] * double(k);
      hp.dtab[k] = d;
      hp.dtab_hi[k] = float(d);
      hp.dtab_lo[k] = float(d - double(hp.dtab_hi[k]));
    }
  }
  if (has_device(c)) {
    int st = need_device(c);
    if (st != MCD_OK) return st;
    if (!c->d_eps) {
      cudaError_t er = cudaMallocAsync(&c->d_eps, sizeof(double) * kMaxSites, c->stream);
      if (er == cudaSuccess) er = cudaMallocAsync(&c->d_U, sizeof(double) * kMaxSites, c->stream);
      if (er != cudaSuccess) return cuda_fail(c, er, "cudaMalloc(eps, U)");
    }
    cudaError_t er = cudaMemcpyAsync(c->d_eps, e.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
    if (er == cudaSuccess)
      er = cudaMemcpyAsync(c->d_U, u.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
    if (er == cudaSuccess) er = cudaStreamSynchronize(c->stream);   // e, u are locals
    if (er != cudaSuccess) return cuda_fail(c, er, "copy eps, U");
    hp.eps = c->d_eps;
    hp.U = c->d_U;
    // partner classes for the single-column kernel (n <= 16), built inside
    // each amplitude class so that every partner class has one amplitude
    hp.n_pcls = 0;
    hp.ptab = nullptr;
    if (n <= 16 && hp.n_class > 0) {
      std::vector<std::array<int, 16>> first;   // first[c][i] = partner or -1
      std::vector<double> amp;
      bool ok = true;
      int b = 0;
      for (int ac = 0; ac < hp.n_class && ok; ++ac) {
        const size_t c0 = first.size();
        for (; b < hp.cls_end[ac]; ++b) {
          const int u = __builtin_ctz(hp.bonds[b].mask);
          const int v = 31 - __builtin_clz(hp.bonds[b].mask);
          bool placed = false;
          for (size_t cc = c0; cc < first.size() && !placed; ++cc) {
            if (first[cc][u] < 0) { first[cc][u] = v; placed = true; }
            else if (first[cc][v] < 0) { first[cc][v] = u; placed = true; }
          }
          if (!placed) {
            if (int(first.size()) == kMaxPClasses) { ok = false; break; }
            std::array<int, 16> f;
            f.fill(-1);
            f[u] = v;
            first.push_back(f);
            amp.push_back(hp.cls_t[ac]);
          }
        }
      }
      if (ok && !first.empty()) {
        const int np = int(first.size());
        const int ng = (np + 3) / 4;
        std::vector<uint2> tab(size_t(ng) * 512 + size_t(np) * 16);
        for (auto& e : tab) e = make_uint2(0u, 0u);
        uint2* flips = tab.data() + size_t(ng) * 512;
        for (int cc = 0; cc < np; ++cc) {
          uint32_t fm = 0;
          uint64_t pk = 0;
          for (int i = 0; i < 16; ++i) {
            const int j = first[cc][i];
            if (j < 0) continue;
            fm |= 1u << i;
            pk |= uint64_t(j) << (4 * i);
            {
              const int lo = std::min(i, j), hi = std::max(i, j);
              flips[size_t(cc) * 16 + i] =
                  make_uint2((1u << i) | (1u << j), ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u));
            }
            const int k = j >> 3, bit = j & 7;
            const int g = cc / 4, slot = cc % 4;
            for (int vv = 0; vv < 256; ++vv) {
              if (!((vv >> bit) & 1)) continue;
              uint2& e = tab[size_t(g) * 512 + size_t(k) * 256 + vv];
              const uint32_t add = (1u << i) << (16 * (slot & 1));
              if (slot < 2) e.x |= add; else e.y |= add;
            }
          }
          hp.pfirst[cc] = fm;
          hp.ppart[cc] = pk;
          hp.pcls_t[cc] = amp[cc];
          hp.pcls_hi[cc] = float(amp[cc]);
          hp.pcls_lo[cc] = float(amp[cc] - double(hp.pcls_hi[cc]));
        }
        if (c->d_pclass) cudaFreeAsync(c->d_pclass, c->stream);
        c->d_pclass = nullptr;
        cudaError_t er2 = cudaMallocAsync(&c->d_pclass, tab.size() * sizeof(uint2), c->stream);
        if (er2 == cudaSuccess)
          er2 = cudaMemcpyAsync(c->d_pclass, tab.data(), tab.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                                c->stream);
        if (er2 == cudaSuccess) er2 = cudaStreamSynchronize(c->stream);   // tab is a local
        if (er2 != cudaSuccess) return cuda_fail(c, er2, "partner tables");
        hp.ptab = static_cast<const uint2*>(c->d_pclass);
        hp.pflip = hp.ptab + size_t(ng) * 512;
        hp.n_pcls = np;
      }
    }
  }
  c->has_ham = true;
  cache_invalidate(c->idx.A);   // records hold classes and signs of this Hamiltonian's bonds
  cache_invalidate(c->idx.B);
  if (sector_changed) {
    c->basis.clear();
    c->n_basis = 0;
    if (has_device(c)) free_index(c->idx, c->stream);
    free_lanczos(c->lw);
  }
  c->idx.nnz = -1;
  return MCD_OK;
}

int mcd_build_basis(mcd_ctx* c, uint64_t seed, int64_t n_target, double beta, const uint64_t* seed_states,
                    int64_t n_seed, int flags, int64_t* n_out) {
  if (!c) return MCD_E_INVALID;
  if (!c->has_ham) return fail(c, MCD_E_STATE, "no Hamiltonian set");
  if (!seed_states || n_seed < 1) return fail(c, MCD_E_INVALID, "at least one seed state is required");
  if (!(beta >= 0.0) || !std::isfinite(beta)) return fail(c, MCD_E_INVALID, "beta must be finite and >= 0");
  if (flags & ~MCD_SAMPLE_NEW_ONLY) return fail(c, MCD_E_INVALID, "unknown sampler flag");
  if (n_target < 1 || double(n_target) > sector_size(c->n, c->n_up, c->n_dn))
    return fail(c, MCD_E_INVALID, "n_target must be in [1, sector size]");
  if (n_target > 0x7FFFFFFF) return fail(c, MCD_E_INVALID, "n_target above 2^31 - 1");
  const bool dev_ok = has_device(c) && device_sampler_eligible(c);
  if (c->sampler_where == 2 && !dev_ok)
    return fail(c, MCD_E_INVALID,
                has_device(c) ? "device sampler needs every nonzero U_i equal" : "device sampler needs a device");
  if (dev_ok && c->sampler_where != 1) {
    int st = need_device(c);
    if (st != MCD_OK) return st;
    st = sample_basis_device(c, seed, n_target, beta, seed_states, n_seed, flags, n_out);
    if (st == MCD_W_SHORT) c->err = "sampler stopped early: no new states";
    return st;
  }
  std::vector<uint64_t> F;
  int st;
  try {
    st = sample_basis(c, seed, n_target, beta, seed_states, n_seed, flags, F);
  } catch (const std::bad_alloc&) {
    return fail(c, MCD_E_OOM, "sampler: out of host memory");
  }
  if (st < 0) return st;
  int st2 = install_basis(c, std::move(F));
  if (st2 != MCD_OK) return st2;
  if (n_out) *n_out = c->n_basis;
  if (st == MCD_W_SHORT) c->err = "sampler stopped early: no new states";
  return st;
}

int mcd_set_basis(mcd_ctx* c, const uint64_t* w, int64_t n) {
  if (!c) return MCD_E_INVALID;
  if (!c->has_ham) return fail(c, MCD_E_STATE, "no Hamiltonian set");
  if (!w || n < 1) return fail(c, MCD_E_INVALID, "basis must hold at least one word");
  if (n > 0x7FFFFFFF) return fail(c, MCD_E_INVALID, "basis above 2^31 - 1 states");
  if (has_device(c)) {
    // straight to the device: the index build checks order and sector there
    int st = need_device(c);
    if (st != MCD_OK) return st;
    c->basis.clear();
    c->basis_on_host = false;
    c->n_basis = 0;
    c->gs_valid = false;
    st = build_index(c, w, n, false);
    if (st != MCD_OK) return st;
    c->n_basis = n;
    return MCD_OK;
  }
  const int ns = c->n;
  const uint64_t half = ns == 32 ? 0xFFFFFFFFull : ((1ull << ns) - 1);
  for (int64_t k = 0; k < n; ++k) {
    if (k > 0 && w[k] <= w[k - 1]) return fail(c, MCD_E_INVALID, "basis words must be strictly ascending");
    if (ns < 32 && (w[k] >> (2 * ns)) != 0) return fail(c, MCD_E_SECTOR, "word has bits above 2*n_sites");
    if (__builtin_popcountll(w[k] >> ns) != c->n_up || __builtin_popcountll(w[k] & half) != c->n_dn)
      return fail(c, MCD_E_SECTOR, "word outside the (N_up, N_dn) sector");
  }
  std::vector<uint64_t> v;
  try {
    v.assign(w, w + n);
  } catch (const std::bad_alloc&) {
    return fail(c, MCD_E_OOM, "out of host memory");
  }
  return install_basis(c, std::move(v));
}

int mcd_set_basis_device(mcd_ctx* c, const uint64_t* w, int64_t n) {
  if (!c) return MCD_E_INVALID;
  if (!c->has_ham) return fail(c, MCD_E_STATE, "no Hamiltonian set");
  int st = need_device(c);
  if (st != MCD_OK) return st;
  if (!w || n < 1) return fail(c, MCD_E_INVALID, "basis must hold at least one word");
  if (n > 0x7FFFFFFF) return fail(c, MCD_E_INVALID, "basis above 2^31 - 1 states");
  if (reinterpret_cast<uintptr_t>(w) % 8) return fail(c, MCD_E_INVALID, "misaligned words");
  c->basis.clear();
  c->basis_on_host = false;
  c->n_basis = 0;
  c->gs_valid = false;
  st = build_index(c, w, n, true);
  if (st != MCD_OK) return st;
  c->n_basis = n;
  return MCD_OK;
}

int mcd_get_basis(const mcd_ctx* cc, uint64_t* out, int64_t cap, int64_t* n) {
  if (!cc || !n) return MCD_E_INVALID;
  mcd_ctx* c = const_cast<mcd_ctx*>(cc);
  *n = c->n_basis;
  if (!out || cap <= 0 || c->n_basis == 0) return MCD_OK;
  const int64_t k = std::min<int64_t>(cap, *n);
  if (c->basis_on_host) {
    std::memcpy(out, c->basis.data(), sizeof(uint64_t) * size_t(k));
    return MCD_OK;
  }
  int st = need_device(c);
  if (st != MCD_OK) return st;
  cudaError_t e = cudaMemcpyAsync(out, c->idx.words, sizeof(uint64_t) * size_t(k), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "copy basis to host");
}

int mcd_launch_count(const mcd_ctx* c, int64_t* n) {
  if (!c || !n) return MCD_E_INVALID;
  *n = c->launches;
  return MCD_OK;
}

int mcd_basis_info(mcd_ctx* c, int64_t* n_states, int64_t* n_up_blocks, int64_t* n_dn_blocks,
                   int64_t* nnz) {
  if (!c) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  if (n_states) *n_states = c->n_basis;
  if (!has_device(c)) {
    if (n_up_blocks || n_dn_blocks || nnz) return fail(c, MCD_E_NODEVICE, "index lives on the device");
    return MCD_OK;
  }
  if (n_up_blocks) *n_up_blocks = c->idx.A.nblk;
  if (n_dn_blocks) *n_dn_blocks = c->idx.B.nblk;
  if (nnz) {
    if (c->idx.nnz < 0) {
      st = need_device(c);
      if (st != MCD_OK) return st;
      int64_t v = 0;
      st = hv_connections(c, nullptr, nullptr, nullptr, 0, &v);
      if (st != MCD_OK) return st;
    }
    *nnz = c->idx.nnz;
  }
  return MCD_OK;
}

int mcd_hv_cache_info(mcd_ctx* c, int64_t* bytes, int64_t* n_conn, int* rec_bytes, int* wait_errors) {
  if (!c) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  const ConnCache& A = c->idx.A.cc;
  const ConnCache& B = c->idx.B.cc;
  const bool ok = has_device(c) && A.valid && B.valid;
  if (bytes) *bytes = ok ? (A.n_groups + B.n_groups) * 256 : 0;
  if (n_conn) *n_conn = ok ? A.n_conn + B.n_conn : 0;
  if (rec_bytes) *rec_bytes = ok ? A.rec_bytes : 0;
  if (wait_errors) {
    unsigned int v = 0;
    if (ok) {
      st = cache_errors(c, &v);
      if (st != MCD_OK) return st;
    }
    *wait_errors = v ? 1 : 0;
  }
  return MCD_OK;
}

int mcd_apply(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype) {
  if (!c) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  if ((st = need_device(c)) != MCD_OK) return st;
  if (!x || !y) return fail(c, MCD_E_INVALID, "null vector");
  if (dtype != MCD_F64 && dtype != MCD_F32) return fail(c, MCD_E_INVALID, "dtype must be MCD_F64 or MCD_F32");
  if (ncols < 1 || ld < ncols) return fail(c, MCD_E_INVALID, "need 1 <= ncols <= ld");
  const size_t es = dtype == MCD_F64 ? 8 : 4;
  const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
  const uintptr_t bytes = uintptr_t(c->idx.n) * uintptr_t(ld) * es;
  if (xa < ya + bytes && ya < xa + bytes) return fail(c, MCD_E_INVALID, "x and y overlap");
  if (xa % es || ya % es) return fail(c, MCD_E_INVALID, "misaligned vector");
  st = hv_apply(c, x, y, ncols, ld, dtype, nullptr, 0);
  if (st != MCD_OK || !c->apply_sync) return st;
  return take_wait_errors(c);
}

int mcd_hv_adjoint(mcd_ctx* c, const void* u, const void* v, int ncols, int ld, int dtype, double* grad_t,
                   double* grad_eps, double* grad_U) {
  if (!c) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  if ((st = need_device(c)) != MCD_OK) return st;
  if (!u || !v) return fail(c, MCD_E_INVALID, "null vector");
  if (dtype != MCD_F64 && dtype != MCD_F32) return fail(c, MCD_E_INVALID, "dtype must be MCD_F64 or MCD_F32");
  if (ncols < 1 || ld < ncols) return fail(c, MCD_E_INVALID, "need 1 <= ncols <= ld");
  return hv_adjoint(c, u, v, ncols, ld, dtype, grad_t, grad_eps, grad_U);
}

int mcd_diagonal(mcd_ctx* c, double* diag) {
  if (!c) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  if ((st = need_device(c)) != MCD_OK) return st;
  if (!diag) return fail(c, MCD_E_INVALID, "null output");
  return hv_diagonal(c, diag);
}

int mcd_connections(mcd_ctx* c, int64_t* rows, int64_t* cols, double* vals, int64_t cap, int64_t* nnz) {
  if (!c || !nnz) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  if ((st = need_device(c)) != MCD_OK) return st;
  if (rows && (!cols || !vals)) return fail(c, MCD_E_INVALID, "rows, cols and vals go together");
  return hv_connections(c, rows, cols, vals, cap, nnz);
}

int mcd_lanczos_ground(mcd_ctx* c, int max_iter, double tol, uint64_t seed, int dtype, double* E0, void* psi,
                       int* iters, double* residual) {
  if (!c) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  if ((st = need_device(c)) != MCD_OK) return st;
  if (!E0 || !iters || !residual) return fail(c, MCD_E_INVALID, "null output pointer");
  if (max_iter < 1 || max_iter > 100000) return fail(c, MCD_E_INVALID, "max_iter must be in [1, 100000]");
  if (dtype != MCD_F64 && dtype != MCD_F32) return fail(c, MCD_E_INVALID, "dtype must be MCD_F64 or MCD_F32");
  if (!std::isfinite(tol)) return fail(c, MCD_E_INVALID, "tol must be finite");
  return lanczos_ground(c, max_iter, tol, seed, dtype, E0, psi, iters, residual);
}

int mcd_band_lanczos_green(mcd_ctx* c, const int* site, const int* spin, int L, int n_block_iter, double w_t,
                           int dtype, const double* z_re, const double* z_im, int nz, double* G_re, double* G_im,
                           int64_t* dim_plus, int64_t* dim_minus) {
  if (!c) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  if ((st = need_device(c)) != MCD_OK) return st;
  if (!site || !spin || nz < 0 || (nz > 0 && (!z_re || !z_im || !G_re || !G_im)))
    return fail(c, MCD_E_INVALID, "null argument");
  if (dtype != MCD_F64 && dtype != MCD_F32) return fail(c, MCD_E_INVALID, "dtype must be MCD_F64 or MCD_F32");
  try {
    return band_lanczos_green(c, site, spin, L, n_block_iter, w_t, dtype, z_re, z_im, nz, G_re, G_im, dim_plus,
                              dim_minus);
  } catch (const std::bad_alloc&) {
    return fail(c, MCD_E_OOM, "band Lanczos: out of host memory");
  }
}

int mcd_green_gradient(mcd_ctx* c, const int* site, const int* spin, int L, int n_block_iter, double w_t,
                       const double* z_re, const double* z_im, int nz, const double* g_re, const double* g_im,
                       double cg_tol, double* grad_t, double* grad_eps, double* grad_U, int* cg_iters) {
  if (!c) return MCD_E_INVALID;
  int st = need_basis(c);
  if (st != MCD_OK) return st;
  if ((st = need_device(c)) != MCD_OK) return st;
  if (!site || !spin || nz < 1 || !z_re || !z_im || !g_re || !g_im || !grad_t || !grad_eps || !grad_U)
    return fail(c, MCD_E_INVALID, "null argument");
  if (!(cg_tol > 0.0 && cg_tol < 1.0)) return fail(c, MCD_E_INVALID, "cg_tol must be in (0, 1)");
  try {
    return green_gradient(c, site, spin, L, n_block_iter, w_t, z_re, z_im, nz, g_re, g_im, grad_t, grad_eps, grad_U,
                          cg_tol, cg_iters);
  } catch (const std::bad_alloc&) {
    return fail(c, MCD_E_OOM, "Green gradient: out of host memory");
  }
}

int mcd_batch_band_lanczos_green(mcd_ctx* const* ctxs, int n_inst, const int* site, const int* spin, int L,
                                 int n_block_iter, double w_t, int dtype, const double* z_re, const double* z_im,
                                 int nz, double* G_re, double* G_im, int64_t* dim_plus, int64_t* dim_minus) {
  int st = check_instances(ctxs, n_inst, false);
  if (st != MCD_OK) return st;
  if (nz < 0 || (nz > 0 && (!G_re || !G_im))) return fail(ctxs[0], MCD_E_INVALID, "null argument");
  const size_t per = size_t(nz) * size_t(std::max(L, 0)) * size_t(std::max(L, 0));
  return run_instances(ctxs, n_inst, [&](int i, mcd_ctx* c) {
    return mcd_band_lanczos_green(c, site, spin, L, n_block_iter, w_t, dtype, z_re, z_im, nz,
                                  G_re ? G_re + per * i : nullptr, G_im ? G_im + per * i : nullptr,
                                  dim_plus ? dim_plus + i : nullptr, dim_minus ? dim_minus + i : nullptr);
  });
}

int mcd_batch_green_gradient(mcd_ctx* const* ctxs, int n_inst, const int* site, const int* spin, int L,
                             int n_block_iter, double w_t, const double* z_re, const double* z_im, int nz,
                             const double* g_re, const double* g_im, double cg_tol, double* grad_t,
                             double* grad_eps, double* grad_U, int* cg_iters) {
  int st = check_instances(ctxs, n_inst, true);
  if (st != MCD_OK) return st;
  if (!g_re || !g_im || !grad_t || !grad_eps || !grad_U || nz < 1)
    return fail(ctxs[0], MCD_E_INVALID, "null argument");
  const int n = ctxs[0]->n;
  const size_t per = size_t(nz) * size_t(std::max(L, 0)) * size_t(std::max(L, 0));
  return run_instances(ctxs, n_inst, [&](int i, mcd_ctx* c) {
    return mcd_green_gradient(c, site, spin, L, n_block_iter, w_t, z_re, z_im, nz, g_re + per * i, g_im + per * i,
                              cg_tol, grad_t + size_t(n) * n * i, grad_eps + size_t(n) * i, grad_U + size_t(n) * i,
                              cg_iters ? cg_iters + i : nullptr);
  });
}

int mcd_symeig(int n, const double* A, double* w, int rows, double* X) {
  if (n < 0 || (n > 0 && (!A || !w)) || rows < 0) return MCD_E_INVALID;
  if (n == 0) return MCD_OK;
  std::vector<double> work(A, A + size_t(n) * n);
  return symeig_leading(n, work.data(), w, X ? rows : 0, X) == 0 ? MCD_OK : MCD_E_NOT_CONVERGED;
}

int mcd_batch_apply(mcd_ctx* const* ctxs, int n_inst, const void* x, void* y, int dtype) {
  try {
    return batch_apply(ctxs, n_inst, x, y, dtype);
  } catch (const std::bad_alloc&) {
    return ctxs && n_inst > 0 && ctxs[0] ? fail(ctxs[0], MCD_E_OOM, "batch: out of host memory") : MCD_E_OOM;
  }
}

int mcd_batch_lanczos_ground(mcd_ctx* const* ctxs, int n_inst, int max_iter, double tol, uint64_t seed, int dtype,
                             double* E0, int* iters, double* residual, void* const* psi) {
  if (ctxs && n_inst > 0 && ctxs[0] && ctxs[0]->batch_mode == 0) {
    // every instance's own solve, concurrently: each records its E0, steps and
    // residual; the first failing instance's status (e.g. MCD_E_NOT_CONVERGED)
    // is returned with every instance's outputs written
    int st = check_instances(ctxs, n_inst, false);
    if (st != MCD_OK) return st;
    if (!E0) return fail(ctxs[0], MCD_E_INVALID, "batch Lanczos arguments");
    return run_instances(ctxs, n_inst, [&](int i, mcd_ctx* c) {
      int it = 0;
      double r = 0.0;
      c->keep_gs = true;   // as the lockstep form, every instance keeps its ground state
      const int s = mcd_lanczos_ground(c, max_iter, tol, seed, dtype, E0 + i, psi ? psi[i] : nullptr, &it, &r);
      c->keep_gs = false;
      if (iters) iters[i] = it;
      if (residual) residual[i] = r;
      if (s == MCD_E_NOT_CONVERGED) return fail(c, s, "Lanczos: residual above tol after max_iter steps");
      return s;
    });
  }
  try {
    return batch_lanczos_ground(ctxs, n_inst, max_iter, tol, seed, dtype, E0, iters, residual, psi);
  } catch (const std::bad_alloc&) {
    return ctxs && n_inst > 0 && ctxs[0] ? fail(ctxs[0], MCD_E_OOM, "batch: out of host memory") : MCD_E_OOM;
  }
}

int mcd_lanczos_coeffs(const mcd_ctx* c, double* a, double* b, int cap, int* m) {
  if (!c || !m) return MCD_E_INVALID;
  *m = int(c->last_a.size());
  const int k = std::min(cap, *m);
  for (int i = 0; i < k; ++i) {
    if (a) a[i] = c->last_a[i];
    if (b) b[i] = c->last_b[i];
  }
  return MCD_OK;
}

int mcd_kernel_times(mcd_ctx* c, double* ms, int64_t* count, int n_classes, int reset) {
  if (!c) return MCD_E_INVALID;
  if (n_classes < 0) return fail(c, MCD_E_INVALID, "n_classes < 0");
  if (c->tm) {
    timing_collect(c);
    for (int i = 0; i < n_classes && i < kTimingClasses; ++i) {
      if (ms) ms[i] = c->tm->ms[i];
      if (count) count[i] = c->tm->count[i];
    }
    if (reset)
      for (int i = 0; i < kTimingClasses; ++i) {
        c->tm->ms[i] = 0;
        c->tm->count[i] = 0;
      }
  } else {
    for (int i = 0; i < n_classes && i < kTimingClasses; ++i) {
      if (ms) ms[i] = 0;
      if (count) count[i] = 0;
    }
  }
  return MCD_OK;
}

}  // extern "C"
