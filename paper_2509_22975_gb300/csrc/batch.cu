// Batched H~v and Lanczos ground states of many small Hamiltonians.
//
// Embedding calculations solve many impurity models at once (one
// Hamiltonian, one Monte Carlo basis per instance, bases of uneven size).
// Here every instance keeps its own context (Hamiltonian, basis, two-layout
// index, Eq. (1) and App. B exactly as for one model); a batch gathers the
// instances' index pointers and Hamiltonians in device tables and runs
//   - H~v (pass B, then pass A with the fused <x, y>) as persistent kernels
//     that pull (instance, work item) units from a device counter, so uneven
//     instances load-balance across the GPU; each CTA reloads the bond table
//     only when the instance changes; lookups by the per-block shared bitmap
//     (n_sites <= 16);
//   - the Lanczos recursion of App. B in its normalised form for all
//     instances in lockstep: one launch per phase for the whole batch,
//     per-instance scalars on the device, per-instance reductions in a fixed
//     order (deterministic), instances that converged or broke down frozen by
//     a device flag;
//   - the launches of a chunk of steps captured once in a CUDA graph and
//     replayed (the kernels read the step number from device memory, so the
//     graph does not change between chunks);
//   - the persistent grid size picked by timing the candidates on the first
//     batch of a given size (autotuning), remembered per size class.
// The fp32 form ends, like the single-instance one, with the fp64 Rayleigh
// quotient of each instance's Ritz vector.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "hv_common.cuh"

namespace mcd {
namespace {

constexpr int kBT = 256;
constexpr int kBWarps = kBT / 32;
constexpr uint64_t kGammaB = 0x9E3779B97F4A7C15ull;
constexpr int kMaxInst = 1 << 16;

__host__ __device__ __forceinline__ uint64_t bmix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct BInst {
  Layout A, B;
  int64_t off;           // first element of the instance in batch vectors
  int64_t n;
  const HamParams* hp;   // device copy
  int item0[2];          // first work item of the instance in the B / A lists
  int nitem[2];
};

struct BItem {
  int inst;
  int item;              // work item of the instance's layout (kItem states)
  int part;              // part of the item (its states split in `split` equal runs)
};

struct BArgs {
  const BInst* inst;
  const BItem* items;
  int n_items;
  int* counter;          // work-queue head (zeroed before each launch)
  const void* x;         // x of instance i: x + step * xstride + off_i
  int64_t xstride;
  void* y;               // y of instance i: y + off_i
  const int* step;       // device step number (nullptr: 0)
  const int* active;     // per-instance flag (nullptr: all)
  double* partials;      // per work item <x, y> (pass A)
  int nw;                // bitmap words (2^nmax / 32)
  int xs_cap;            // elements of staged x
  int split;             // parts per work item (the tile size is kItem / split states)
};

// Persistent H~v pass over all instances' work items, one column.
template <typename T, bool PASS_A, bool DOT>
__global__ void __launch_bounds__(kBT) batch_hv_kernel(const BArgs a) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint32_t* bm = reinterpret_cast<uint32_t*>(s_dyn);
  uint16_t* pre = reinterpret_cast<uint16_t*>(bm + a.nw);
  T* xs = reinterpret_cast<T*>(s_dyn + ((size_t(a.nw) * 6 + 15) & ~size_t(15)));
  __shared__ uint32_t s_mask[kMaxBonds], s_betw[kMaxBonds];
  __shared__ float s_thi[kMaxBonds], s_tlo[kMaxBonds];
  __shared__ double s_t64[kMaxBonds];
  __shared__ int s_nb, s_uniform, s_nsites, s_item, s_loaded;
  __shared__ double s_dtab[kMaxSites + 1];
  __shared__ float s_dhi[kMaxSites + 1], s_dlo[kMaxSites + 1];
  __shared__ const double* s_eps;
  __shared__ const double* s_U;
  __shared__ double s_red[kBWarps];
  for (int i = threadIdx.x; i < a.nw; i += kBT) bm[i] = 0u;
  if (threadIdx.x == 0) s_loaded = -1;
  const int step = a.step ? *a.step : 0;
  const int lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();   // s_item and the bitmap of the previous item are free
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int ii = s_item;
    if (ii >= a.n_items) break;
    const BItem bi = a.items[ii];
    if (a.active && !a.active[bi.inst]) {
      if (DOT && threadIdx.x == 0) a.partials[ii] = 0.0;
      continue;
    }
    const BInst& ins = a.inst[bi.inst];
    if (bi.inst != s_loaded) {
      const HamParams* hp = ins.hp;
      const int nb = hp->n_bonds;
      for (int b = threadIdx.x; b < nb; b += kBT) {
        s_mask[b] = hp->bonds[b].mask;
        s_betw[b] = hp->bonds[b].between;
        s_thi[b] = hp->bonds[b].t_hi;
        s_tlo[b] = hp->bonds[b].t_lo;
        s_t64[b] = hp->bonds[b].t;
      }
      if (threadIdx.x <= kMaxSites) {
        s_dtab[threadIdx.x] = hp->dtab[threadIdx.x];
        s_dhi[threadIdx.x] = hp->dtab_hi[threadIdx.x];
        s_dlo[threadIdx.x] = hp->dtab_lo[threadIdx.x];
      }
      __syncthreads();   // every thread has read s_loaded before it changes
      if (threadIdx.x == 0) {
        s_nb = nb;
        s_uniform = hp->uniform;
        s_nsites = hp->n_sites;
        s_eps = hp->eps;
        s_U = hp->U;
        s_loaded = bi.inst;
      }
      __syncthreads();
    }
    const Layout L = PASS_A ? ins.A : ins.B;
    const int nb = s_nb, ns = s_nsites;
    const T* x = static_cast<const T*>(a.x) + int64_t(step) * a.xstride + ins.off;
    T* y = static_cast<T*>(a.y) + ins.off;
    // the states of this part of the work item, and the blocks they lie in
    const int64_t ki0 = int64_t(bi.item) * kItem;
    const int64_t ki1 = (ki0 + kItem < L.n) ? ki0 + kItem : L.n;
    const int64_t chunk = (ki1 - ki0 + a.split - 1) / a.split;
    const int64_t k0 = (ki0 + bi.part * chunk < ki1) ? ki0 + bi.part * chunk : ki1;
    const int64_t k1 = (k0 + chunk < ki1) ? k0 + chunk : ki1;
    if (k0 >= k1) {
      if (DOT && threadIdx.x == 0) a.partials[ii] = 0.0;
      continue;
    }
    uint32_t b0 = L.item_blk[bi.item];
    while (int64_t(L.blk_off[b0 + 1]) <= k0) ++b0;
    uint32_t b1 = b0;
    while (int64_t(b1) + 1 < L.nblk && int64_t(L.blk_off[b1 + 1]) < k1) ++b1;
    double dot_acc = 0.0;
    for (uint32_t blk = b0; blk <= b1; ++blk) {
      const int bs = int(L.blk_off[blk]), be = int(L.blk_off[blk + 1]);
      const uint32_t major = L.blk_major[blk];
      const int bsz = be - bs;
      const bool staged = bsz <= a.xs_cap;
      for (int q = threadIdx.x; q < bsz; q += kBT) {
        const uint32_t d = L.minor[bs + q];
        atomicOr(&bm[d >> 5], 1u << (d & 31));
        if (q == 0 || (L.minor[bs + q - 1] >> 5) != (d >> 5)) pre[d >> 5] = uint16_t(q);
        if (staged) xs[q] = x[PASS_A ? int64_t(bs + q) : int64_t(L.perm[bs + q])];
      }
      __syncthreads();
      const int lo = (int64_t(bs) > k0) ? bs : int(k0);
      const int hi = (int64_t(be) < k1) ? be : int(k1);
      for (int k = lo + threadIdx.x; k < hi; k += kBT) {
        const uint32_t m = L.minor[k];
        Acc<T> acc;
        acc.zero();
        for (int b = 0; b < nb; ++b) {
          const uint32_t mk = s_mask[b];
          if (__popc(m & mk) != 1) continue;
          const uint32_t m2 = m ^ mk;
          const uint32_t wd = bm[m2 >> 5];
          const uint32_t bit = m2 & 31u;
          if (!((wd >> bit) & 1u)) continue;
          const int q = int(pre[m2 >> 5]) + __popc(wd & ((1u << bit) - 1u));
          const T xv = staged ? xs[q] : x[PASS_A ? int64_t(bs + q) : int64_t(L.perm[bs + q])];
          const bool neg = __popc(m & s_betw[b]) & 1;
          if (sizeof(T) == 4) acc.fma(neg ? -T(s_thi[b]) : T(s_thi[b]), neg ? -T(s_tlo[b]) : T(s_tlo[b]), xv);
          else acc.fma(neg ? -T(s_t64[b]) : T(s_t64[b]), T(0), xv);
        }
        if (PASS_A) {
          const T xk = staged ? xs[k - bs] : x[k];
          T dh, dl;
          if (s_uniform) {
            const int nu = __popc(major & m);
            dh = sizeof(T) == 4 ? T(s_dhi[nu]) : T(s_dtab[nu]);
            dl = sizeof(T) == 4 ? T(s_dlo[nu]) : T(0);
          } else {
            double d = 0.0;
            for (int i = 0; i < ns; ++i) {
              const int u = (major >> i) & 1, v = (m >> i) & 1;
              d += s_eps[i] * double(u + v) + s_U[i] * double(u & v);
            }
            dh = T(d);
            dl = sizeof(T) == 4 ? T(d - double(dh)) : T(0);
          }
          acc.fma(dh, dl, xk);
          const T out = acc.value() + y[k];
          y[k] = out;
          if (DOT) dot_acc += double(xk) * double(out);
        } else {
          y[L.perm[k]] = acc.value();
        }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < bsz; q += kBT) bm[L.minor[bs + q] >> 5] = 0u;
      __syncthreads();   // cleared before the next block sets bits
    }
    if (DOT) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dot_acc += __shfl_xor_sync(0xffffffffu, dot_acc, o);
      if (lane == 0) s_red[threadIdx.x >> 5] = dot_acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < kBWarps; ++w) sum += s_red[w];
        a.partials[ii] = sum;
      }
    }
  }
}

// instance of element k (offsets[n_inst] = total), binary search
__device__ __forceinline__ int inst_of(const int64_t* off, int n_inst, int64_t k) {
  int lo = 0, len = n_inst;
  while (len > 1) {
    const int half = len >> 1;
    if (off[lo + half] <= k) lo += half;
    len -= half;
  }
  return lo;
}

// fixed-order block sum; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* s_red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kBWarps; ++w) t += s_red[w];
  __syncthreads();
  return t;
}

// per-instance start vectors s_0 (slot 0) and |s_0|^2; grid = n_inst
template <typename T>
__global__ void __launch_bounds__(kBT) bstart_kernel(T* V, const int64_t* off, uint64_t key, double* nrm2, int cap) {
  __shared__ double s_red[kBWarps];
  const int i = blockIdx.x;
  const int64_t a = off[i], b = off[i + 1];
  double acc = 0.0;
  for (int64_t k = a + threadIdx.x; k < b; k += kBT) {
    const uint64_t r = bmix(key ^ uint64_t(k - a));
    const T v = T(double(r >> 11) * 0x1p-53 * 2.0 - 1.0);
    V[k] = v;
    acc += double(v) * double(v);
  }
  const double t = block_sum(acc, s_red);
  if (threadIdx.x == 0) nrm2[int64_t(i) * cap] = t;
}

// dot[i][step] = sum of the instance's pass-A item partials, in item order
// (split parts per work item: the instance's parts are contiguous)
__global__ void bdot_kernel(const BInst* inst, int n_inst, const double* partials, const int* step, double* dot,
                            int cap, const int* active, int split) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst || !active[i]) return;
  double s = 0.0;
  const int64_t t0 = int64_t(split) * inst[i].item0[1], t1 = t0 + int64_t(split) * inst[i].nitem[1];
  for (int64_t t = t0; t < t1; ++t) s += partials[t];
  dot[int64_t(i) * cap + *step] = s;
}

// s_{n+1} = sig_n w - a_n sig_n s_n - b_n sig_{n-1} s_{n-1}, per instance
template <typename T>
__global__ void __launch_bounds__(kBT) bupdate_kernel(T* V, const T* W, int64_t ntot, const int64_t* off, int n_inst,
                                                     const double* nrm2, const double* dot, int cap, const int* step,
                                                     const int* active) {
  __shared__ int64_t s_off[1024 + 1];
  const int st = *step;
  const bool small = n_inst <= 1024;
  if (small)
    for (int i = threadIdx.x; i <= n_inst; i += kBT) s_off[i] = off[i];
  __syncthreads();
  const T* s = V + int64_t(st) * ntot;
  const T* sp = V + int64_t(st > 0 ? st - 1 : 0) * ntot;
  T* o = V + int64_t(st + 1) * ntot;
  for (int64_t k = int64_t(blockIdx.x) * kBT + threadIdx.x; k < ntot; k += int64_t(gridDim.x) * kBT) {
    const int i = inst_of(small ? s_off : off, n_inst, k);
    if (!active[i]) continue;
    const double nn = nrm2[int64_t(i) * cap + st];
    const double sig = 1.0 / sqrt(nn);
    const double al = sig, be = -(dot[int64_t(i) * cap + st] / nn) * sig;
    T v = T(al) * W[k] + T(be) * s[k];
    if (st > 0) v += T(-sqrt(nn) / sqrt(nrm2[int64_t(i) * cap + st - 1])) * sp[k];
    o[k] = v;
  }
}

// nrm2[i][step + 1] = |s_{step+1}|^2 of instance i; grid = n_inst; then the
// last block advances the step counter
template <typename T>
__global__ void __launch_bounds__(kBT) bnorm_kernel(const T* V, int64_t ntot, const int64_t* off, double* nrm2, int cap,
                                                   int* step, const int* active, unsigned int* ticket) {
  __shared__ double s_red[kBWarps];
  const int i = blockIdx.x;
  const int st = *step;
  if (active[i]) {
    const T* o = V + int64_t(st + 1) * ntot;
    double acc = 0.0;
    for (int64_t k = off[i] + threadIdx.x; k < off[i + 1]; k += kBT) acc += double(o[k]) * double(o[k]);
    const double t = block_sum(acc, s_red);
    if (threadIdx.x == 0) nrm2[int64_t(i) * cap + st + 1] = t;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ticket, 1u) == gridDim.x - 1) {
      *ticket = 0u;
      *step = st + 1;
    }
  }
}

// psi64 of every instance = sum_j coef[i][j] s_j: fp64 for fp64 vectors,
// double-float (df_fma, coefficients as (hi, lo) floats) for fp32 vectors
__global__ void bcombine_kernel(double* psi, const double* V, int64_t ntot, const int64_t* off, int n_inst,
                                const double* coef, const int* m, int cap) {
  for (int64_t k = int64_t(blockIdx.x) * kBT + threadIdx.x; k < ntot; k += int64_t(gridDim.x) * kBT) {
    const int i = inst_of(off, n_inst, k);
    double acc = 0.0;
    for (int j = 0; j < m[i]; ++j) acc = fma(coef[int64_t(i) * cap + j], V[int64_t(j) * ntot + k], acc);
    psi[k] = acc;
  }
}
__global__ void bcombine32_kernel(double* psi, const float* V, int64_t ntot, const int64_t* off, int n_inst,
                                  const float2* coef, const int* m, int cap) {
  for (int64_t k = int64_t(blockIdx.x) * kBT + threadIdx.x; k < ntot; k += int64_t(gridDim.x) * kBT) {
    const int i = inst_of(off, n_inst, k);
    float h = 0.f, l = 0.f;
    for (int j = 0; j < m[i]; ++j) {
      const float2 c = coef[int64_t(i) * cap + j];
      df_fma(h, l, c.x, c.y, V[int64_t(j) * ntot + k]);
    }
    psi[k] = double(h) + double(l);
  }
}

// out[i] = <a, b> over instance i (grid = n_inst)
__global__ void __launch_bounds__(kBT) bdot64_kernel(const double* a, const double* b, const int64_t* off,
                                                    double* out) {
  __shared__ double s_red[kBWarps];
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int64_t k = off[i] + threadIdx.x; k < off[i + 1]; k += kBT) acc += a[k] * b[k];
  const double t = block_sum(acc, s_red);
  if (threadIdx.x == 0) out[i] = t;
}

template <typename T>
__global__ void bcast_kernel(T* out, const double* v, int64_t n, const double* scale_of_inst, const int64_t* off,
                             int n_inst) {
  for (int64_t k = int64_t(blockIdx.x) * kBT + threadIdx.x; k < n; k += int64_t(gridDim.x) * kBT)
    out[k] = T(v[k] * scale_of_inst[inst_of(off, n_inst, k)]);
}

int egrid(int64_t n) { return int(std::max<int64_t>(1, std::min<int64_t>((n + kBT - 1) / kBT, int64_t(device_sms()) * 16))); }

struct DevPtr {
  void* p = nullptr;
  DevPtr() = default;
  DevPtr(const DevPtr&) = delete;
  DevPtr& operator=(const DevPtr&) = delete;
  ~DevPtr() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 8); }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// grid sizes the autotuner tries (CTAs per SM) and its memory, per size class
const int kGridCand[] = {2, 4, 8};
const int kSplitCand[] = {1, 2, 4};   // parts per work item: tiles of kItem, kItem / 2, kItem / 4 states
constexpr int kNSplit = 3;
std::mutex g_tune_mu;
struct Tuned {
  int cps = 2;     // CTAs per SM
  int split = 1;   // parts per work item
};
std::map<std::pair<int, int>, Tuned> g_tuned;   // (log2 total, log2 n_inst) -> grid and tile

class Batch {
 public:
  Batch(mcd_ctx* const* ctxs, int n) : c0_(ctxs[0]), n_(n), ctxs_(ctxs, ctxs + n) {}
  ~Batch() {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    if (s_) cudaStreamDestroy(s_);
  }

  int setup() {
    cudaError_t e = cudaSetDevice(c0_->device);
    for (int i = 0; i < n_ && e == cudaSuccess; ++i) e = cudaStreamSynchronize(ctxs_[i]->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch stream");
    std::vector<BInst> inst(n_);
    std::vector<BItem> items[2];
    off_.assign(n_ + 1, 0);
    nmax_ = 1;
    for (int i = 0; i < n_; ++i) {
      mcd_ctx* c = ctxs_[i];
      inst[i].A = c->idx.A;
      inst[i].B = c->idx.B;
      inst[i].off = off_[i];
      inst[i].n = c->idx.n;
      off_[i + 1] = off_[i] + c->idx.n;
      nmax_ = std::max(nmax_, c->n);
      for (int p = 0; p < 2; ++p) {
        const Layout& L = p ? c->idx.A : c->idx.B;
        inst[i].item0[p] = int(items[p].size());
        inst[i].nitem[p] = int(L.n_items);
        for (int64_t t = 0; t < L.n_items; ++t) items[p].push_back(BItem{i, int(t), 0});
      }
    }
    ntot_ = off_[n_];
    // device copies of the Hamiltonians (each with its own eps/U pointers)
    e = hps_.alloc(sizeof(HamParams) * n_);
    for (int i = 0; i < n_ && e == cudaSuccess; ++i)
      e = cudaMemcpy(hps_.as<HamParams>() + i, ctxs_[i]->hp, sizeof(HamParams), cudaMemcpyHostToDevice);
    for (int i = 0; i < n_; ++i) inst[i].hp = hps_.as<HamParams>() + i;
    if (e == cudaSuccess) e = inst_.alloc(sizeof(BInst) * n_);
    if (e == cudaSuccess) e = cudaMemcpy(inst_.p, inst.data(), sizeof(BInst) * n_, cudaMemcpyHostToDevice);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p)
      for (int si = 0; si < kNSplit && e == cudaSuccess; ++si) {
        const int sp = kSplitCand[si];
        std::vector<BItem> parts;
        parts.reserve(items[p].size() * sp);
        for (const BItem& b : items[p])
          for (int q = 0; q < sp; ++q) parts.push_back(BItem{b.inst, b.item, q});
        nitems_[p][si] = int(parts.size());
        e = items_[p][si].alloc(sizeof(BItem) * parts.size());
        if (e == cudaSuccess)
          e = cudaMemcpy(items_[p][si].p, parts.data(), sizeof(BItem) * parts.size(), cudaMemcpyHostToDevice);
      }
    if (e == cudaSuccess) e = offd_.alloc(sizeof(int64_t) * (n_ + 1));
    if (e == cudaSuccess) e = cudaMemcpy(offd_.p, off_.data(), sizeof(int64_t) * (n_ + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = counters_.alloc(sizeof(int) * 2 + sizeof(unsigned int) + sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(counters_.p, 0, sizeof(int) * 2 + sizeof(unsigned int) + sizeof(int));
    if (e == cudaSuccess) e = partials_.alloc(sizeof(double) * std::max(nitems_[1][kNSplit - 1], 1));
    if (e == cudaSuccess) e = active_.alloc(sizeof(int) * n_);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch tables");
    std::vector<int> ones(n_, 1);
    e = cudaMemcpy(active_.p, ones.data(), sizeof(int) * n_, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch flags");
    nw_ = nmax_ >= 5 ? (1 << (nmax_ - 5)) : 1;
    return MCD_OK;
  }

  int* counter(int p) const { return counters_.as<int>() + p; }
  unsigned int* ticket() const { return reinterpret_cast<unsigned int*>(counters_.as<int>() + 2); }
  int* step() const { return counters_.as<int>() + 3; }

  template <typename T>
  size_t smem_bytes() const {
    return ((size_t(nw_) * 6 + 15) & ~size_t(15)) + size_t(xs_cap<T>()) * sizeof(T);
  }
  template <typename T>
  int xs_cap() const {
    return int(24 * 1024 / sizeof(T));
  }

  // one H~v pair: x + step*xstride -> y over all instances (dot: fused <x, y>)
  template <typename T>
  cudaError_t hv(const T* x, int64_t xstride, const int* stepp, T* y, bool dot, Tuned tc) {
    const int ctas_per_sm = tc.cps;
    int si = 0;
    while (si + 1 < kNSplit && kSplitCand[si] != tc.split) ++si;
    BArgs a{};
    a.inst = inst_.as<BInst>();
    a.x = x;
    a.xstride = xstride;
    a.y = y;
    a.step = stepp;
    a.active = active_.as<int>();
    a.partials = partials_.as<double>();
    a.nw = nw_;
    a.xs_cap = xs_cap<T>();
    a.split = kSplitCand[si];
    const size_t smem = smem_bytes<T>();
    static std::atomic<bool> configured{false};
    if (!configured) {
      cudaFuncSetAttribute(batch_hv_kernel<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      cudaFuncSetAttribute(batch_hv_kernel<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      cudaFuncSetAttribute(batch_hv_kernel<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      configured = true;
    }
    for (int p = 0; p < 2; ++p) {
      a.items = items_[p][si].as<BItem>();
      a.n_items = nitems_[p][si];
      a.counter = counter(p);
      cudaError_t e = cudaMemsetAsync(counter(p), 0, sizeof(int), s_);
      if (e != cudaSuccess) return e;
      const int grid = std::max(1, std::min(nitems_[p][si], device_sms() * ctas_per_sm));
      if (p == 0)
        batch_hv_kernel<T, false, false><<<grid, kBT, smem, s_>>>(a);
      else if (dot)
        batch_hv_kernel<T, true, true><<<grid, kBT, smem, s_>>>(a);
      else
        batch_hv_kernel<T, true, false><<<grid, kBT, smem, s_>>>(a);
      MCD_LAUNCHED(c0_);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }

  // persistent grid size and work-unit (tile) size for this batch:
  // remembered per size class, else timed over every candidate pair; the
  // first context's MCD_OPT_BATCH_SPLIT (when set) fixes the tile
  template <typename T>
  Tuned tune(const T* x, T* y) {
    int lt = 0, li = 0;
    while ((int64_t(1) << lt) < ntot_) ++lt;
    while ((1 << li) < n_) ++li;
    const int forced = c0_->batch_split;
    if (!forced) {
      std::lock_guard<std::mutex> g(g_tune_mu);
      auto it = g_tuned.find({lt, li});
      if (it != g_tuned.end()) return it->second;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Tuned best;
    float best_ms = 1e30f;
    for (int sp : kSplitCand) {
      if (forced && sp != forced) continue;
      for (int cand : kGridCand) {
        const Tuned tc{cand, sp};
        hv<T>(x, 0, nullptr, y, false, tc);   // warm-up
        cudaEventRecord(e0, s_);
        for (int r = 0; r < 3; ++r) hv<T>(x, 0, nullptr, y, false, tc);
        cudaEventRecord(e1, s_);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = tc;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!forced) {
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tuned[{lt, li}] = best;
    }
    return best;
  }

  template <typename T>
  int apply(const T* x, T* y) {
    cudaError_t e = sync_from(c0_->stream);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch apply");
    const Tuned cps = tune<T>(x, y);
    e = hv<T>(x, 0, nullptr, y, false, cps);
    if (e == cudaSuccess) e = sync_to(c0_->stream);
    return e == cudaSuccess ? MCD_OK : cuda_fail(c0_, e, "batch apply");
  }

  template <typename T>
  int lanczos(int max_iter, double tol, uint64_t seed, double* E0, int* iters, double* resid, void* const* psi);

 private:
  cudaError_t sync_from(cudaStream_t other) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, other);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_, ev, 0);
    cudaEventDestroy(ev);
    return e;
  }
  cudaError_t sync_to(cudaStream_t other) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, s_);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(other, ev, 0);
    cudaEventDestroy(ev);
    return e;
  }

  mcd_ctx* c0_;
  int n_;
  std::vector<mcd_ctx*> ctxs_;
  std::vector<int64_t> off_;
  int64_t ntot_ = 0;
  int nmax_ = 1, nw_ = 1;
  int nitems_[2][kNSplit] = {};
  cudaStream_t s_ = nullptr;
  DevPtr hps_, inst_, items_[2][kNSplit], offd_, counters_, partials_, active_;
  cudaGraphExec_t graph_exec_ = nullptr;
};

template <typename T>
int Batch::lanczos(int max_iter, double tol, uint64_t seed, double* E0, int* iters, double* resid,
                   void* const* psi) {
  const int cap = max_iter + 2;
  const bool fp32 = sizeof(T) == 4;
  DevPtr V, W, scal, psi64, hpsi, coef, mdev, dots, scale;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  if (double(max_iter + 1) * double(ntot_) * sizeof(T) > 0.8 * double(free_b))
    return fail(c0_, MCD_E_OOM, "batch Lanczos: the Krylov vectors of all instances do not fit");
  cudaError_t e = V.alloc(size_t(max_iter + 1) * ntot_ * sizeof(T));
  if (e == cudaSuccess) e = W.alloc(size_t(ntot_) * sizeof(T));
  if (e == cudaSuccess) e = scal.alloc(sizeof(double) * 2 * size_t(cap) * n_);
  if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Lanczos workspace");
  double* nrm2 = scal.as<double>();
  double* dot = nrm2 + size_t(cap) * n_;
  e = sync_from(c0_->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(scal.p, 0, sizeof(double) * 2 * size_t(cap) * n_, s_);
  if (e == cudaSuccess) e = cudaMemsetAsync(step(), 0, sizeof(int), s_);
  if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Lanczos start");
  const Tuned cps = tune<T>(V.as<T>(), W.as<T>());
  const uint64_t key = bmix(bmix(seed + kGammaB) ^ 0x4C414E43ull);   // same stream as one instance
  bstart_kernel<T><<<n_, kBT, 0, s_>>>(V.as<T>(), offd_.as<int64_t>(), key, nrm2, cap);
  MCD_LAUNCHED(c0_);
  // one Lanczos step for every active instance (all reads of the step number
  // happen on the device, so the same launches serve every step)
  auto enqueue_step = [&]() -> cudaError_t {
    cudaError_t er = hv<T>(V.as<T>(), ntot_, step(), W.as<T>(), true, cps);
    if (er != cudaSuccess) return er;
    bdot_kernel<<<(n_ + 127) / 128, 128, 0, s_>>>(inst_.as<BInst>(), n_, partials_.as<double>(), step(), dot, cap,
                                                 active_.as<int>(), cps.split);
    MCD_LAUNCHED(c0_);
    bupdate_kernel<T><<<egrid(ntot_), kBT, 0, s_>>>(V.as<T>(), W.as<T>(), ntot_, offd_.as<int64_t>(), n_, nrm2, dot,
                                                    cap, step(), active_.as<int>());
    MCD_LAUNCHED(c0_);
    bnorm_kernel<T><<<n_, kBT, 0, s_>>>(V.as<T>(), ntot_, offd_.as<int64_t>(), nrm2, cap, step(), active_.as<int>(),
                                        ticket());
    MCD_LAUNCHED(c0_);
    return cudaGetLastError();
  };
  const int chunk = 16;
  // capture a chunk of steps once (captured launches are counted when the
  // graph is launched)
  cudaGraph_t graph = nullptr;
  const int64_t counted = c0_->launches;
  e = cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal);
  for (int k = 0; k < chunk && e == cudaSuccess; ++k) e = enqueue_step();
  cudaError_t e2 = cudaStreamEndCapture(s_, &graph);
  const int64_t per_graph = c0_->launches - counted;
  c0_->launches = counted;
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&graph_exec_, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Lanczos graph");

  std::vector<int> act(n_, 1), m_of(n_, 0), conv(n_, 0), bad_of(n_, 0);
  std::vector<double> hn(size_t(cap) * n_), hd(size_t(cap) * n_);
  std::vector<std::vector<double>> evs(n_);
  std::vector<double> e0(n_, 0.0), rs(n_, INFINITY);
  int m = 0;
  while (m < max_iter) {
    const int todo = std::min(chunk, max_iter - m);
    if (todo == chunk) {
      e = cudaGraphLaunch(graph_exec_, s_);
      c0_->launches += per_graph;
    } else {
      for (int k = 0; k < todo && e == cudaSuccess; ++k) e = enqueue_step();
    }
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Lanczos step");
    m += todo;
    e = cudaMemcpyAsync(hn.data(), nrm2, sizeof(double) * cap * n_, cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), dot, sizeof(double) * cap * n_, cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Lanczos read-back");
    bool any = false;
    for (int i = 0; i < n_; ++i) {
      if (!act[i]) continue;
      const double* nr = hn.data() + size_t(i) * cap;
      const double* dt = hd.data() + size_t(i) * cap;
      std::vector<double> a(m, 0.0), b(m + 1, 0.0);
      int mm = m;
      bool bad = false, brk = false;
      for (int k = 0; k < m; ++k) {
        a[k] = dt[k] / nr[k];
        if (k > 0) b[k] = std::sqrt(nr[k]);
        if (!std::isfinite(a[k]) || !std::isfinite(b[k])) { mm = k; bad = true; break; }
      }
      b[m] = std::sqrt(nr[m]);
      double sc = 0.0;
      for (int k = 0; k < mm; ++k) sc = std::max(sc, std::fabs(a[k]) + b[k] + b[k + 1]);
      for (int k = 0; k < mm; ++k)
        if (b[k + 1] <= 1e-14 * std::max(1.0, sc) || !std::isfinite(b[k + 1])) {
          mm = k + 1;
          brk = true;
          break;
        }
      if (mm == 0) {
        act[i] = 0;
        bad_of[i] = 1;
        continue;
      }
      evs[i].assign(mm, 0.0);
      e0[i] = tridiag_lowest(a.data(), b.data(), mm, evs[i].data());
      rs[i] = (brk ? 0.0 : b[mm]) * std::fabs(evs[i][mm - 1]);
      m_of[i] = mm;
      if (brk || bad) {
        act[i] = 0;
        conv[i] = brk;
        bad_of[i] = bad && !brk;
      } else if (tol > 0 && rs[i] < tol * std::max(1.0, std::fabs(e0[i]))) {
        act[i] = 0;
        conv[i] = 1;
      }
      any |= act[i] != 0;
    }
    if (!any) break;
    e = cudaMemcpyAsync(active_.p, act.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, s_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Lanczos flags");
  }
  // Ritz vectors (fp64): psi_i = sum_j ev_i[j] sig_j s_j; the fp32 form
  // returns each instance's fp64 Rayleigh quotient
  int status = MCD_OK;
  for (int i = 0; i < n_; ++i) {
    if (bad_of[i]) status = MCD_E_BREAKDOWN;
    else if (!conv[i] && tol > 0 && status == MCD_OK) status = MCD_E_NOT_CONVERGED;
  }
  {
    // the fp64 Ritz vector of every instance: its Rayleigh quotient (fp32
    // form), the caller's psi, and the ground state each context keeps for
    // the Green function (as mcd_lanczos_ground keeps it)
    std::vector<double> cf(size_t(cap) * n_, 0.0);
    for (int i = 0; i < n_; ++i)
      for (int j = 0; j < m_of[i]; ++j) cf[size_t(i) * cap + j] = evs[i][j] / std::sqrt(hn[size_t(i) * cap + j]);
    std::vector<float2> cf32(fp32 ? cf.size() : 0);
    for (size_t k = 0; k < cf32.size(); ++k) cf32[k] = split_coef(cf[k]);
    e = psi64.alloc(sizeof(double) * ntot_);
    if (e == cudaSuccess) e = hpsi.alloc(sizeof(double) * ntot_);
    if (e == cudaSuccess) e = coef.alloc(sizeof(double) * cf.size());
    if (e == cudaSuccess) e = mdev.alloc(sizeof(int) * n_);
    if (e == cudaSuccess) e = dots.alloc(sizeof(double) * 2 * n_);
    if (e == cudaSuccess) e = scale.alloc(sizeof(double) * n_);
    if (e == cudaSuccess)
      e = fp32 ? cudaMemcpyAsync(coef.p, cf32.data(), sizeof(float2) * cf32.size(), cudaMemcpyHostToDevice, s_)
               : cudaMemcpyAsync(coef.p, cf.data(), sizeof(double) * cf.size(), cudaMemcpyHostToDevice, s_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mdev.p, m_of.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, s_);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Ritz vectors");
    if (fp32)
      bcombine32_kernel<<<egrid(ntot_), kBT, 0, s_>>>(psi64.as<double>(), reinterpret_cast<const float*>(V.p), ntot_,
                                                      offd_.as<int64_t>(), n_, coef.as<float2>(), mdev.as<int>(), cap);
    else
      bcombine_kernel<<<egrid(ntot_), kBT, 0, s_>>>(psi64.as<double>(), reinterpret_cast<const double*>(V.p), ntot_,
                                                    offd_.as<int64_t>(), n_, coef.as<double>(), mdev.as<int>(), cap);
    MCD_LAUNCHED(c0_);
    std::vector<int> ones(n_, 1);
    e = cudaMemcpyAsync(active_.p, ones.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, s_);
    if (e == cudaSuccess) e = hv<double>(psi64.as<double>(), 0, nullptr, hpsi.as<double>(), false, cps);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Ritz H psi");
    bdot64_kernel<<<n_, kBT, 0, s_>>>(psi64.as<double>(), psi64.as<double>(), offd_.as<int64_t>(), dots.as<double>());
    bdot64_kernel<<<n_, kBT, 0, s_>>>(psi64.as<double>(), hpsi.as<double>(), offd_.as<int64_t>(),
                                      dots.as<double>() + n_);
    MCD_LAUNCHED(c0_);
    MCD_LAUNCHED(c0_);
    std::vector<double> hdots(2 * n_);
    e = cudaMemcpyAsync(hdots.data(), dots.p, sizeof(double) * 2 * n_, cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Rayleigh quotients");
    std::vector<double> sc(n_);
    for (int i = 0; i < n_; ++i) {
      sc[i] = 1.0 / std::sqrt(hdots[i]);
      if (fp32) e0[i] = hdots[n_ + i] / hdots[i];
    }
    e = cudaMemcpyAsync(scale.p, sc.data(), sizeof(double) * n_, cudaMemcpyHostToDevice, s_);
    if (e != cudaSuccess) return cuda_fail(c0_, e, "batch psi");
    {
      DevPtr g64;
      e = g64.alloc(sizeof(double) * ntot_);
      if (e != cudaSuccess) return cuda_fail(c0_, e, "batch ground states");
      bcast_kernel<double><<<egrid(ntot_), kBT, 0, s_>>>(g64.as<double>(), psi64.as<double>(), ntot_,
                                                         scale.as<double>(), offd_.as<int64_t>(), n_);
      MCD_LAUNCHED(c0_);
      for (int i = 0; i < n_ && e == cudaSuccess; ++i) {
        mcd_ctx* c = ctxs_[i];
        const int64_t ni = off_[i + 1] - off_[i];
        c->gs_valid = false;
        if (!c->gs_psi || c->gs_n != ni) {
          if (c->gs_psi) cudaFreeAsync(c->gs_psi, s_);
          c->gs_psi = nullptr;
          e = cudaMallocAsync(reinterpret_cast<void**>(&c->gs_psi), sizeof(double) * size_t(ni), s_);
          if (e != cudaSuccess) break;
          c->gs_n = ni;
        }
        e = cudaMemcpyAsync(c->gs_psi, g64.as<double>() + off_[i], sizeof(double) * size_t(ni),
                            cudaMemcpyDeviceToDevice, s_);
        c->gs_E0 = e0[i];
        c->gs_valid = !bad_of[i];
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s_);   // g64 is freed on return
      if (e != cudaSuccess) return cuda_fail(c0_, e, "batch ground states");
    }
    if (psi) {
      // normalised Ritz vector of each instance into the caller's buffers
      DevPtr out;
      e = out.alloc(sizeof(T) * ntot_);
      if (e != cudaSuccess) return cuda_fail(c0_, e, "batch psi");
      bcast_kernel<T><<<egrid(ntot_), kBT, 0, s_>>>(out.as<T>(), psi64.as<double>(), ntot_, scale.as<double>(),
                                                    offd_.as<int64_t>(), n_);
      MCD_LAUNCHED(c0_);
      for (int i = 0; i < n_ && e == cudaSuccess; ++i)
        if (psi[i])
          e = cudaMemcpyAsync(psi[i], out.as<T>() + off_[i], sizeof(T) * (off_[i + 1] - off_[i]),
                              cudaMemcpyDeviceToDevice, s_);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
      if (e != cudaSuccess) return cuda_fail(c0_, e, "batch psi copy");
    }
  }
  e = cudaStreamSynchronize(s_);
  if (e == cudaSuccess) e = sync_to(c0_->stream);
  if (e != cudaSuccess) return cuda_fail(c0_, e, "batch Lanczos");
  for (int i = 0; i < n_; ++i) {
    E0[i] = e0[i];
    if (iters) iters[i] = m_of[i];
    if (resid) resid[i] = rs[i];
  }
  return status;
}

// common argument checks; 0 or an error status
int check_batch(mcd_ctx* const* ctxs, int n) {
  if (!ctxs || n < 1 || n > kMaxInst || !ctxs[0]) return MCD_E_INVALID;
  mcd_ctx* c0 = ctxs[0];
  for (int i = 0; i < n; ++i) {
    mcd_ctx* c = ctxs[i];
    if (!c) return fail(c0, MCD_E_INVALID, "batch: null context");
    if (c->device < 0) return fail(c0, MCD_E_NODEVICE, "batch: host-only context");
    if (c->device != c0->device) return fail(c0, MCD_E_INVALID, "batch: contexts on different devices");
    if (!c->has_ham || c->idx.n == 0) return fail(c0, MCD_E_STATE, "batch: context without Hamiltonian or basis");
    if (c->n > 16) return fail(c0, MCD_E_INVALID, "batch: n_sites above 16");
  }
  return MCD_OK;
}

}  // namespace

int batch_apply(mcd_ctx* const* ctxs, int n, const void* x, void* y, int dtype) {
  int st = check_batch(ctxs, n);
  if (st != MCD_OK) return st;
  if (!x || !y || (dtype != MCD_F64 && dtype != MCD_F32)) return fail(ctxs[0], MCD_E_INVALID, "batch apply arguments");
  Batch b(ctxs, n);
  st = b.setup();
  if (st != MCD_OK) return st;
  return dtype == MCD_F64 ? b.apply<double>(static_cast<const double*>(x), static_cast<double*>(y))
                          : b.apply<float>(static_cast<const float*>(x), static_cast<float*>(y));
}

int batch_lanczos_ground(mcd_ctx* const* ctxs, int n, int max_iter, double tol, uint64_t seed, int dtype,
                         double* E0, int* iters, double* resid, void* const* psi) {
  int st = check_batch(ctxs, n);
  if (st != MCD_OK) return st;
  if (!E0 || max_iter < 1 || max_iter > 100000 || !(tol >= 0.0) || (dtype != MCD_F64 && dtype != MCD_F32))
    return fail(ctxs[0], MCD_E_INVALID, "batch Lanczos arguments");
  Batch b(ctxs, n);
  st = b.setup();
  if (st != MCD_OK) return st;
  return dtype == MCD_F64 ? b.lanczos<double>(max_iter, tol, seed, E0, iters, resid, psi)
                          : b.lanczos<float>(max_iter, tol, seed, E0, iters, resid, psi);
}

}  // namespace mcd
