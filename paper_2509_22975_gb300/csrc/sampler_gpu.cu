// Monte Carlo construction of the truncated basis F~ on the device, with the
// same result, bit for bit, as the host sampler (sampler.cpp).
//
// Sec. "Subspace of the ground state": every step applies every hopping term
// to every starting state of the step; a proposed state b is accepted with
// probability min(exp(-beta E_U(b)), 1) (the Boltzmann-factor Eq.); accepted
// states start the next step (the "revisit" reading; MCD_SAMPLE_NEW_ONLY:
// only the new ones), new states join F~ until it holds n_target states.
// The random choices are those of the host sampler: one SplitMix64 draw
//   draw = f(f(f(f(seed + G) ^ step) ^ parent) ^ hop),  hop = s n^2 + i n + j,
// accept iff (draw >> 11) 2^-53 < p; an overshooting last step keeps the new
// states of smallest (f(f(f(seed + G) ^ ~0) ^ word), word).
//
// One step on the device:
//   1. count / scan / write: thread per starting state, accepted children
//      written at scanned offsets (deterministic, no atomics);
//   2. stable LSD radix sort (8-bit digits) of the children, then unique;
//   3. new states = children absent from F~ (binary search in sorted F~);
//   4. overshoot: stable sort of the new states by priority (they are already
//      in word order, so equal priorities stay in word order), first `room`,
//      sorted back by word;
//   5. F~ := merge(F~, new) by ranks (disjoint sorted sets).
// p depends on the double occupancy only through E_U.  The device path takes
// Hamiltonians whose nonzero U_i are all equal (uniform U, or U on a subset of
// sites such as an impurity's cluster): then E_U, summed in site order as the
// host does, depends only on k = number of doubly occupied U-sites, and the
// table p[k] is computed on the host by the host sampler's own formula, so
// no exponential is evaluated on the device.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mcd_internal.h"

namespace mcd {
namespace {

constexpr uint64_t kGammaS = 0x9E3779B97F4A7C15ull;
constexpr int kT = 256;
constexpr int kTileItems = 8;
constexpr int kTile = kT * kTileItems;   // keys per radix tile
constexpr int kDigits = 256;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct DHop {
  uint64_t from, to, flip, id;
};

struct SampleArgs {
  int n;
  int n_hops;
  uint64_t half;     // mask of one spin's n bits
  uint64_t umask;    // sites with U_i != 0
  uint64_t key2;     // f(key1 ^ step)
  double p[kMaxSites + 1];
};

// children of frontier[k] accepted in this step: counted (WRITE = false) or
// written at out[off[k]...] in hop order
template <bool WRITE>
__global__ void propose_kernel(const uint64_t* __restrict__ frontier, int64_t nf, const DHop* __restrict__ hops,
                               const SampleArgs a, uint32_t* cnt, const uint32_t* off, uint64_t* out) {
  __shared__ double s_p[kMaxSites + 1];
  if (threadIdx.x <= kMaxSites) s_p[threadIdx.x] = a.p[threadIdx.x];
  __syncthreads();
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const uint64_t w = frontier[k];
  const uint64_t key3 = mix64(a.key2 ^ w);
  uint32_t c = 0;
  uint64_t* o = WRITE ? out + off[k] : nullptr;
  for (int h = 0; h < a.n_hops; ++h) {
    const uint64_t from = __ldg(&hops[h].from), to = __ldg(&hops[h].to);
    if (!(w & from) || (w & to)) continue;
    const uint64_t child = w ^ __ldg(&hops[h].flip);
    const uint64_t r = mix64(key3 ^ __ldg(&hops[h].id));
    const uint64_t both = (child >> a.n) & child & a.half & a.umask;
    const double u = double(r >> 11) * 0x1p-53;
    if (u < s_p[__popcll(both)]) {
      if (WRITE) o[c] = child;
      ++c;
    }
  }
  if (!WRITE) cnt[k] = c;
}

// ---- stable LSD radix sort of 64-bit keys (optional 64-bit values) ---------------
__global__ void hist64_kernel(const uint64_t* keys, int64_t n, int shift, uint32_t* hist, int64_t ntiles) {
  __shared__ uint32_t h[kDigits];
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kTile;
  for (int k = threadIdx.x; k < kTile; k += blockDim.x)
    if (base + k < n) atomicAdd(&h[(keys[base + k] >> shift) & (kDigits - 1)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) hist[int64_t(d) * ntiles + blockIdx.x] = h[d];
}

// rounds of kT consecutive keys; a key's rank among equal digits comes from
// the lower lanes of its warp and the lower warps, so input order is kept
template <bool VALS>
__global__ void scatter64_kernel(const uint64_t* kin, const uint64_t* vin, int64_t n, int shift, const uint32_t* offs,
                                 int64_t ntiles, uint64_t* kout, uint64_t* vout) {
  constexpr int kWarps = kT / 32;
  __shared__ uint32_t run[kDigits];
  __shared__ uint32_t wc[kWarps][kDigits];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) run[d] = offs[int64_t(d) * ntiles + blockIdx.x];
  const int64_t base = int64_t(blockIdx.x) * kTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kTileItems; ++r) {
    for (int k = threadIdx.x; k < kWarps * kDigits; k += blockDim.x) (&wc[0][0])[k] = 0;
    __syncthreads();
    const int64_t i = base + int64_t(r) * kT + threadIdx.x;
    const bool ok = i < n;
    const uint64_t key = ok ? kin[i] : 0ull;
    const int d = ok ? int((key >> shift) & (kDigits - 1)) : kDigits;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (ok && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      uint32_t pos = run[d] + rank;
      for (int ww = 0; ww < warp; ++ww) pos += wc[ww][d];
      kout[pos] = key;
      if (VALS) vout[pos] = vin[i];
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kDigits; dd += blockDim.x) {
      uint32_t s = 0;
      for (int ww = 0; ww < kWarps; ++ww) s += wc[ww][dd];
      run[dd] += s;
    }
    __syncthreads();
  }
}

__global__ void flag_unique_kernel(const uint64_t* a, int64_t n, uint32_t* flag) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (i == 0 || a[i] != a[i - 1]) ? 1u : 0u;
}

// flag[i] = 1 if a[i] is absent from the sorted F[0, nF)
__global__ void flag_absent_kernel(const uint64_t* a, int64_t n, const uint64_t* F, int64_t nF, uint32_t* flag) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = a[i];
  int64_t lo = 0, len = nF;
  while (len > 0) {
    const int64_t half = len >> 1;
    if (F[lo + half] < key) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  flag[i] = (lo < nF && F[lo] == key) ? 0u : 1u;
}

__global__ void compact_kernel(const uint64_t* a, int64_t n, const uint32_t* flag, const uint32_t* pos, uint64_t* out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) out[pos[i]] = a[i];
}

__global__ void prio_kernel(const uint64_t* a, int64_t n, uint64_t kp, uint64_t* prio) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) prio[i] = mix64(kp ^ a[i]);
}

// out[i + rank of a[i] in b] = a[i]  (a, b sorted, disjoint)
__global__ void merge_rank_kernel(const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb, uint64_t* out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= na) return;
  const uint64_t key = a[i];
  int64_t lo = 0, len = nb;
  while (len > 0) {
    const int64_t half = len >> 1;
    if (b[lo + half] < key) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  out[i + lo] = key;
}

int grid_for(int64_t n) { return int((n + kT - 1) / kT); }

__global__ void sum_counts64_kernel(const uint32_t* a, int64_t n, unsigned long long* out) {
  unsigned long long s = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    s += a[i];
  atomicAdd(out, s);   // integer sums: the order does not matter
}

// Stream-ordered scratch that frees itself.
struct Buf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { reset(); }
  void reset() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

class DevSampler {
 public:
  explicit DevSampler(mcd_ctx* c) : c_(c), s_(c->stream) {}

  cudaError_t alloc(Buf& b, size_t bytes) {
    b.s = s_;
    return cudaMallocAsync(&b.p, bytes ? bytes : 8, s_);
  }

  // stable sort of keys[0, n) (and vals) on the low `bits` bits
  cudaError_t sort(uint64_t* keys, uint64_t* vals, int64_t n, int bits) {
    if (n <= 1) return cudaSuccess;
    const int64_t ntiles = (n + kTile - 1) / kTile;
    if (ntiles * kDigits > 0xFFFFFFFFll) return cudaErrorInvalidValue;
    Buf k2, v2, hist;
    cudaError_t e = alloc(k2, size_t(n) * 8);
    if (e == cudaSuccess && vals) e = alloc(v2, size_t(n) * 8);
    if (e == cudaSuccess) e = alloc(hist, size_t(ntiles) * kDigits * 4);
    if (e != cudaSuccess) return e;
    uint64_t* kin = keys;
    uint64_t* vin = vals;
    uint64_t* kout = k2.as<uint64_t>();
    uint64_t* vout = v2.as<uint64_t>();
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
      hist64_kernel<<<int(ntiles), kT, 0, s_>>>(kin, n, 8 * p, hist.as<uint32_t>(), ntiles);
      MCD_LAUNCHED(c_);
      e = scan_u32(c_, hist.as<uint32_t>(), hist.as<uint32_t>(), ntiles * kDigits, s_);
      if (e != cudaSuccess) return e;
      if (vals)
        scatter64_kernel<true><<<int(ntiles), kT, 0, s_>>>(kin, vin, n, 8 * p, hist.as<uint32_t>(), ntiles, kout, vout);
      else
        scatter64_kernel<false><<<int(ntiles), kT, 0, s_>>>(kin, nullptr, n, 8 * p, hist.as<uint32_t>(), ntiles, kout,
                                                            nullptr);
      MCD_LAUNCHED(c_);
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
    if (kin != keys) {
      e = cudaMemcpyAsync(keys, kin, size_t(n) * 8, cudaMemcpyDeviceToDevice, s_);
      if (e == cudaSuccess && vals) e = cudaMemcpyAsync(vals, vin, size_t(n) * 8, cudaMemcpyDeviceToDevice, s_);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
  }

  // out = a[flag], returns the count
  cudaError_t compact(const uint64_t* a, int64_t n, uint32_t* flag, Buf& out, int64_t& nout) {
    nout = 0;
    if (n == 0) return alloc(out, 8);
    Buf pos;
    cudaError_t e = alloc(pos, size_t(n) * 4);
    if (e == cudaSuccess) e = scan_u32(c_, flag, pos.as<uint32_t>(), n, s_);
    uint32_t last_pos = 0, last_flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last_pos, pos.as<uint32_t>() + n - 1, 4, cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last_flag, flag + n - 1, 4, cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
    if (e != cudaSuccess) return e;
    nout = int64_t(last_pos) + last_flag;
    e = alloc(out, size_t(nout) * 8);
    if (e != cudaSuccess) return e;
    compact_kernel<<<grid_for(n), kT, 0, s_>>>(a, n, flag, pos.as<uint32_t>(), out.as<uint64_t>());
    MCD_LAUNCHED(c_);
    return cudaGetLastError();
  }

 private:
  mcd_ctx* c_;
  cudaStream_t s_;
};

}  // namespace

int sort_unique_device(mcd_ctx* c, uint64_t* keys, int64_t n, int bits, uint64_t** out, int64_t* nout) {
  *out = nullptr;
  *nout = 0;
  DevSampler ds(c);
  cudaStream_t s = c->stream;
  cudaError_t e = ds.sort(keys, nullptr, n, bits);
  if (e != cudaSuccess) return cuda_fail(c, e, "sort of words");
  Buf flag, uniq;
  e = ds.alloc(flag, size_t(std::max<int64_t>(n, 1)) * 4);
  if (e == cudaSuccess && n > 0) {
    flag_unique_kernel<<<grid_for(n), kT, 0, s>>>(keys, n, flag.as<uint32_t>());
    MCD_LAUNCHED(c);
    e = cudaGetLastError();
  }
  int64_t nu = 0;
  if (e == cudaSuccess) e = ds.compact(keys, n, flag.as<uint32_t>(), uniq, nu);
  if (e != cudaSuccess) return cuda_fail(c, e, "unique words");
  *out = uniq.as<uint64_t>();
  uniq.p = nullptr;   // the caller frees it (stream-ordered)
  *nout = nu;
  return MCD_OK;
}

bool device_sampler_eligible(const mcd_ctx* c) {
  double u = 0.0;
  for (int i = 0; i < c->n; ++i) {
    if (c->U[i] == 0.0) continue;
    if (u == 0.0) u = c->U[i];
    else if (c->U[i] != u) return false;
  }
  return true;
}

int sample_basis_device(mcd_ctx* c, uint64_t seed, int64_t n_target, double beta, const uint64_t* seeds,
                        int64_t n_seed, int flags, int64_t* n_out) {
  const int n = c->n;
  cudaStream_t s = c->stream;
  DevSampler ds(c);
  SampleArgs a{};
  a.n = n;
  a.half = (n == 32) ? 0xFFFFFFFFull : ((1ull << n) - 1);
  a.umask = 0;
  for (int i = 0; i < n; ++i)
    if (c->U[i] != 0.0) a.umask |= 1ull << i;
  // p[k]: the host sampler's min(exp(-beta E_U), 1) for k doubly occupied
  // U-sites, E_U summed over the sites in order (zero-U sites add nothing)
  for (int k = 0; k <= n; ++k) {
    double e = 0.0;
    int left = k;
    for (int i = 0; i < n && left > 0; ++i)
      if ((a.umask >> i) & 1) {
        e += c->U[i];
        --left;
      }
    const double p = std::exp(-beta * e);
    a.p[k] = p < 1.0 ? p : 1.0;
  }
  std::vector<DHop> hops;
  for (int sp = 0; sp < 2; ++sp) {
    const int shift = (sp == 0) ? n : 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        if (i == j || c->t[size_t(i) * n + j] == 0.0) continue;
        DHop h;
        h.from = 1ull << (j + shift);
        h.to = 1ull << (i + shift);
        h.flip = h.from | h.to;
        h.id = uint64_t(sp) * n * n + uint64_t(i) * n + j;
        hops.push_back(h);
      }
  }
  a.n_hops = int(hops.size());
  std::vector<uint64_t> F0(seeds, seeds + n_seed);
  std::sort(F0.begin(), F0.end());
  F0.erase(std::unique(F0.begin(), F0.end()), F0.end());
  for (uint64_t w : F0) {
    if (n < 32 && (w >> (2 * n)) != 0) return fail(c, MCD_E_SECTOR, "seed word has bits above 2*n_sites");
    if (__builtin_popcountll(w >> n) != c->n_up || __builtin_popcountll(w & a.half) != c->n_dn)
      return fail(c, MCD_E_SECTOR, "seed word outside the (N_up, N_dn) sector");
  }
  if (int64_t(F0.size()) > n_target) return fail(c, MCD_E_INVALID, "more seed states than n_target");
  const int bits = 2 * n;

  Buf dhops, F, frontier;
  cudaError_t e = ds.alloc(dhops, hops.size() * sizeof(DHop));
  if (e == cudaSuccess && !hops.empty())
    e = cudaMemcpyAsync(dhops.p, hops.data(), hops.size() * sizeof(DHop), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = ds.alloc(F, F0.size() * 8);
  if (e == cudaSuccess) e = cudaMemcpyAsync(F.p, F0.data(), F0.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = ds.alloc(frontier, F0.size() * 8);
  if (e == cudaSuccess) e = cudaMemcpyAsync(frontier.p, F0.data(), F0.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // F0 and hops die with this frame's host vectors
  if (e != cudaSuccess) return cuda_fail(c, e, "device sampler setup");
  int64_t nF = int64_t(F0.size()), nfr = nF;
  const uint64_t key1 = mix64(seed + kGammaS);
  uint64_t step = 0;
  int stagnant = 0;
  int status = MCD_OK;
  while (nF < n_target) {
    ++step;
    a.key2 = mix64(key1 ^ step);
    // 1. proposals
    Buf cnt, off, kids;
    int64_t nk = 0;
    e = ds.alloc(cnt, size_t(nfr) * 4);
    if (e == cudaSuccess) e = ds.alloc(off, size_t(nfr) * 4);
    if (e != cudaSuccess) break;
    propose_kernel<false><<<grid_for(nfr), kT, 0, s>>>(frontier.as<uint64_t>(), nfr, dhops.as<DHop>(), a,
                                                      cnt.as<uint32_t>(), nullptr, nullptr);
    MCD_LAUNCHED(c);
    {
      // the offsets are 32-bit: when the bound allows more, count exactly first
      if (double(nfr) * double(a.n_hops) >= 4294967295.0) {
        Buf tot;
        unsigned long long h = 0;
        e = ds.alloc(tot, 8);
        if (e == cudaSuccess) e = cudaMemsetAsync(tot.p, 0, 8, s);
        if (e == cudaSuccess) {
          sum_counts64_kernel<<<device_sms() * 4, kT, 0, s>>>(cnt.as<uint32_t>(), nfr, tot.as<unsigned long long>());
          MCD_LAUNCHED(c);
          e = cudaMemcpyAsync(&h, tot.p, 8, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        if (h >= 4294967295ull) {
          status = fail(c, MCD_E_OOM, "device sampler: 2^32 or more accepted proposals in one step");
          break;
        }
      }
      e = scan_u32(c, cnt.as<uint32_t>(), off.as<uint32_t>(), nfr, s);
      uint32_t lo = 0, lc = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&lo, off.as<uint32_t>() + nfr - 1, 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&lc, cnt.as<uint32_t>() + nfr - 1, 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      nk = int64_t(lo) + lc;
    }
    e = ds.alloc(kids, size_t(nk) * 8);
    if (e != cudaSuccess) break;
    if (nk > 0) {
      propose_kernel<true><<<grid_for(nfr), kT, 0, s>>>(frontier.as<uint64_t>(), nfr, dhops.as<DHop>(), a, nullptr,
                                                       off.as<uint32_t>(), kids.as<uint64_t>());
      MCD_LAUNCHED(c);
    }
    // 2. sort + unique = the accepted set
    e = ds.sort(kids.as<uint64_t>(), nullptr, nk, bits);
    if (e != cudaSuccess) break;
    Buf flag, accepted;
    int64_t na = 0;
    e = ds.alloc(flag, size_t(std::max<int64_t>(nk, 1)) * 4);
    if (e != cudaSuccess) break;
    if (nk > 0) {
      flag_unique_kernel<<<grid_for(nk), kT, 0, s>>>(kids.as<uint64_t>(), nk, flag.as<uint32_t>());
      MCD_LAUNCHED(c);
    }
    e = ds.compact(kids.as<uint64_t>(), nk, flag.as<uint32_t>(), accepted, na);
    if (e != cudaSuccess) break;
    kids.reset();
    // 3. new states
    Buf flag2, fresh;
    int64_t nfresh = 0;
    e = ds.alloc(flag2, size_t(std::max<int64_t>(na, 1)) * 4);
    if (e != cudaSuccess) break;
    if (na > 0) {
      flag_absent_kernel<<<grid_for(na), kT, 0, s>>>(accepted.as<uint64_t>(), na, F.as<uint64_t>(), nF,
                                                    flag2.as<uint32_t>());
      MCD_LAUNCHED(c);
    }
    e = ds.compact(accepted.as<uint64_t>(), na, flag2.as<uint32_t>(), fresh, nfresh);
    if (e != cudaSuccess) break;
    // 4. overshoot: keep the `room` new states of smallest (priority, word)
    const int64_t room = n_target - nF;
    if (nfresh > room) {
      Buf prio;
      e = ds.alloc(prio, size_t(nfresh) * 8);
      if (e != cudaSuccess) break;
      prio_kernel<<<grid_for(nfresh), kT, 0, s>>>(fresh.as<uint64_t>(), nfresh, mix64(key1 ^ ~0ull),
                                                  prio.as<uint64_t>());
      MCD_LAUNCHED(c);
      e = ds.sort(prio.as<uint64_t>(), fresh.as<uint64_t>(), nfresh, 64);
      if (e == cudaSuccess) e = ds.sort(fresh.as<uint64_t>(), nullptr, room, bits);
      if (e != cudaSuccess) break;
      nfresh = room;
    }
    // 5. F := merge(F, fresh)
    Buf merged;
    e = ds.alloc(merged, size_t(nF + nfresh) * 8);
    if (e != cudaSuccess) break;
    merge_rank_kernel<<<grid_for(nF), kT, 0, s>>>(F.as<uint64_t>(), nF, fresh.as<uint64_t>(), nfresh,
                                                 merged.as<uint64_t>());
    MCD_LAUNCHED(c);
    if (nfresh > 0) {
      merge_rank_kernel<<<grid_for(nfresh), kT, 0, s>>>(fresh.as<uint64_t>(), nfresh, F.as<uint64_t>(), nF,
                                                       merged.as<uint64_t>());
      MCD_LAUNCHED(c);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    std::swap(F.p, merged.p);
    nF += nfresh;
    stagnant = nfresh == 0 ? stagnant + 1 : 0;
    const bool none_accepted = na == 0;
    if (flags & MCD_SAMPLE_NEW_ONLY) {
      std::swap(frontier.p, fresh.p);
      nfr = nfresh;
    } else {
      std::swap(frontier.p, accepted.p);
      nfr = na;
    }
    if (nF >= n_target) break;
    if (none_accepted || nfr == 0 || stagnant >= 64) {
      status = MCD_W_SHORT;
      break;
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "device sampler");
  if (status < 0) return status;
  c->basis.clear();
  c->basis_on_host = false;
  c->n_basis = 0;
  c->gs_valid = false;
  const int st = build_index(c, F.as<uint64_t>(), nF, true);
  if (st != MCD_OK) return st;
  c->n_basis = nF;
  if (n_out) *n_out = nF;
  return status;
}

}  // namespace mcd
