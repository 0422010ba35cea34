// Lanczos ground state (App. B) on the device.
//
// The recursion phi_{n+1} = H phi_n - a_n phi_n - b_n^2 phi_{n-1} of App. B is
// run in its normalised form: with unit vectors v_n,
//   r = H v_n - a_n v_n - b_n v_{n-1},  a_n = <v_n|H|v_n>,  b_{n+1} = |r|,
// the same tridiagonal H_eff (a_n on the diagonal, b_n beside it).  To avoid
// a separate normalisation pass, the stored vector is s_n = r (unnormalised)
// and v_n = s_n / |s_n|: the H*v pass computes w = H s_n and, fused in its
// last kernel, <s_n, w>; one update kernel then writes
//   s_{n+1} = sig_n w - a_n sig_n s_n - b_n sig_{n-1} s_{n-1}   (sig = 1/|s|)
// over s_{n-1} in place and reduces |s_{n+1}|^2.  Scalars stay on the device
// (fp64); the host reads them every few steps to solve the tridiagonal
// eigenproblem (fp64) and test convergence.  All reductions have a fixed
// order, so a second pass regenerates bit-identical vectors to form the Ritz
// vector sum_n |n><n|Omega_eff> (change-of-basis Eq. of App. B) without
// storing the Krylov basis.
#include <cmath>
#include <vector>

#include "hv_common.cuh"
#include "mcd_internal.h"

namespace mcd {
namespace {

constexpr int kThreads = 256;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// scalar area layout: [0, cap) nrm2[n] = |s_n|^2 ; [cap, 2cap) dotraw[n] = <s_n, H s_n>;
// [2cap] misc reductions
struct Slots {
  int cap;
  __host__ __device__ int nrm2(int n) const { return n; }
  __host__ __device__ int dot(int n) const { return cap + n; }
  __host__ __device__ int misc(int k) const { return 2 * cap + k; }
};

__host__ __device__ __forceinline__ uint64_t smix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Block sum of v; the last CTA to arrive sums the per-CTA partials in a fixed
// order and stores the total to *out.
__device__ void grid_sum(double v, double* partials, unsigned int* ticket, double* out) {
  __shared__ double s_red[kThreads / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += s_red[w];
    partials[blockIdx.x] = s;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < int(gridDim.x); i += kThreads) s += __ldcg(partials + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if (lane == 0) s_red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
    *out = t;
    *ticket = 0u;
  }
}

template <typename T>
struct V4;
template <>
struct V4<float> {
  using type = float4;
  static constexpr int W = 4;
};
template <>
struct V4<double> {
  using type = double2;
  static constexpr int W = 2;
};

__device__ __forceinline__ void ld(const float* p, float* v) {
  float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void st(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void ld(const double* p, double* v) {
  double2 q = *reinterpret_cast<const double2*>(p);
  v[0] = q.x; v[1] = q.y;
}
__device__ __forceinline__ void st(double* p, const double* v) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// sum of squares of W stored values (in T)
template <typename T, int W>
__device__ __forceinline__ T sumsq(const T* v) {
  T s = T(0);
#pragma unroll
  for (int i = 0; i < W; ++i) s = v[i] * v[i] + s;
  return s;
}

// a thread's running sum of such partials: fp64 for fp64 vectors, double-float
// (df_add) for fp32 vectors, so that no fp64 arithmetic runs per element
template <typename T>
struct RunSum;
template <>
struct RunSum<float> {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float x) { df_add(h, l, x); }
  __device__ __forceinline__ double value() const { return double(h) + double(l); }
};
template <>
struct RunSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

// s_0[k] = uniform[-1, 1) from SplitMix64(key ^ k) ; nrm2[0] = |s_0|^2
template <typename T>
__global__ void __launch_bounds__(kThreads) start_kernel(T* s0, int64_t n, uint64_t key, double* partials,
                                                         unsigned int* ticket, double* out) {
  double acc = 0.0;
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads) {
    const uint64_t r = smix(key ^ uint64_t(k));
    const double u = double(r >> 11) * 0x1p-53 * 2.0 - 1.0;
    const T v = T(u);
    s0[k] = v;
    acc += double(v) * double(v);
  }
  grid_sum(acc, partials, ticket, out);
}

// s_next = al * w + be * s + ga * s_prev (written over s_prev), nrm2 reduced.
template <typename T>
__global__ void __launch_bounds__(kThreads) update_kernel(const T* __restrict__ w, const T* __restrict__ s,
                                                          const T* s_prev, T* out, int64_t n, int step,
                                                          const double* scal, Slots sl, double* partials,
                                                          unsigned int* ticket) {
  __shared__ T c_al, c_be, c_ga;
  __shared__ int s_use_prev;
  if (threadIdx.x == 0) {
    const double nn = scal[sl.nrm2(step)];
    const double sig = 1.0 / sqrt(nn);
    const double a = scal[sl.dot(step)] / nn;
    double ga = 0.0;
    if (step > 0) ga = -sqrt(nn) / sqrt(scal[sl.nrm2(step - 1)]);   // -b_n sig_{n-1}
    c_al = T(sig);
    c_be = T(-a * sig);
    c_ga = T(ga);
    s_use_prev = step > 0;
  }
  __syncthreads();
  const T al = c_al, be = c_be, ga = c_ga;
  const bool use_prev = s_use_prev;
  constexpr int W = V4<T>::W;
  RunSum<T> acc;
  const int64_t nv = n / W;
  for (int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x; q < nv; q += int64_t(gridDim.x) * kThreads) {
    T a[W], b[W], c[W], o[W];
    ld(w + q * W, a);
    ld(s + q * W, b);
    if (use_prev) ld(s_prev + q * W, c);
#pragma unroll
    for (int i = 0; i < W; ++i) o[i] = use_prev ? (al * a[i] + be * b[i] + ga * c[i]) : (al * a[i] + be * b[i]);
    st(out + q * W, o);
    acc.add(sumsq<T, W>(o));
  }
  // tail
  if (blockIdx.x == 0) {
    for (int64_t k = nv * W + threadIdx.x; k < n; k += kThreads) {
      T o = al * w[k] + be * s[k];
      if (use_prev) o += ga * s_prev[k];
      out[k] = o;
      acc.add(o * o);
    }
  }
  grid_sum(acc.value(), partials, ticket, const_cast<double*>(scal) + sl.nrm2(step + 1));
}

// psi += coef * s
template <typename T>
__global__ void axpy_kernel(T* psi, const T* s, int64_t n, double coef) {
  const T c = T(coef);
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads)
    psi[k] += c * s[k];
}

// psi[k] = sum_{j < m} coef[j] V[j][k] in fp64 (V: m stored fp64 vectors, stride ld)
__global__ void combine_kernel(double* psi, const double* V, int64_t n, int64_t ld, int m, const double* coef) {
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads) {
    double acc = 0.0;
    for (int j = 0; j < m; ++j) acc = fma(__ldg(coef + j), V[int64_t(j) * ld + k], acc);
    psi[k] = acc;
  }
}

// The same sum over fp32 vectors in double-float (df_fma, coefficients split
// as (hi, lo) floats), written out as double(h) + double(l): four positions
// per thread (16-byte loads; ld is a multiple of 4 and V 16-byte aligned),
// four vectors' loads issued before their arithmetic; the last n % 4
// positions one by one.
__global__ void __launch_bounds__(kThreads) combine32_kernel(double* psi, const float* __restrict__ V, int64_t n,
                                                             int64_t ld, int m, const float2* __restrict__ coef) {
  const int64_t nv = n / 4;
  for (int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x; q < nv; q += int64_t(gridDim.x) * kThreads) {
    float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
    const float* vq = V + 4 * q;
    int j = 0;
    for (; j + 4 <= m; j += 4) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldcs(reinterpret_cast<const float4*>(vq + int64_t(j + u) * ld));
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 c = __ldg(coef + j + u);
        df_fma(h[0], l[0], c.x, c.y, v[u].x);
        df_fma(h[1], l[1], c.x, c.y, v[u].y);
        df_fma(h[2], l[2], c.x, c.y, v[u].z);
        df_fma(h[3], l[3], c.x, c.y, v[u].w);
      }
    }
    for (; j < m; ++j) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(vq + int64_t(j) * ld));
      const float2 c = __ldg(coef + j);
      df_fma(h[0], l[0], c.x, c.y, v.x);
      df_fma(h[1], l[1], c.x, c.y, v.y);
      df_fma(h[2], l[2], c.x, c.y, v.z);
      df_fma(h[3], l[3], c.x, c.y, v.w);
    }
    double2* out = reinterpret_cast<double2*>(psi + 4 * q);
    out[0] = make_double2(double(h[0]) + double(l[0]), double(h[1]) + double(l[1]));
    out[1] = make_double2(double(h[2]) + double(l[2]), double(h[3]) + double(l[3]));
  }
  if (blockIdx.x == 0)
    for (int64_t k = nv * 4 + threadIdx.x; k < n; k += kThreads) {
      float h = 0.f, l = 0.f;
      for (int j = 0; j < m; ++j) {
        const float2 c = __ldg(coef + j);
        df_fma(h, l, c.x, c.y, V[int64_t(j) * ld + k]);
      }
      psi[k] = double(h) + double(l);
    }
}

// psi64 += coef * s (fp64 vectors)
__global__ void axpy64_kernel(double* psi, const double* s, int64_t n, double coef) {
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads)
    psi[k] = fma(coef, s[k], psi[k]);
}

// one term of combine32_kernel's sum when the vectors are regenerated: the
// double-float state (h, l) of each position is kept in psi's own 8 bytes
__global__ void axpy_df_kernel(float2* acc, const float* s, int64_t n, float chi, float clo) {
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads) {
    float2 a = acc[k];
    df_fma(a.x, a.y, chi, clo, s[k]);
    acc[k] = a;
  }
}

// psi[k] = double(h) + double(l) in place of the state (h, l) at the same 8 bytes
__global__ void finish_df_kernel(double* psi, int64_t n) {
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads) {
    const float2 a = reinterpret_cast<const float2*>(psi)[k];
    psi[k] = double(a.x) + double(a.y);
  }
}

// out[k] = T(v[k] * f)
template <typename T>
__global__ void cast_scale_kernel(T* out, const double* v, int64_t n, double f) {
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads)
    out[k] = T(v[k] * f);
}

// out = sum_k a[k] b[k] (or sum a^2 when b == nullptr)
template <typename T>
__global__ void __launch_bounds__(kThreads) dot_kernel(const T* a, const T* b, int64_t n, double* partials,
                                                       unsigned int* ticket, double* out) {
  double acc = 0.0;
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads)
    acc += double(a[k]) * double(b ? b[k] : a[k]);
  grid_sum(acc, partials, ticket, out);
}

// out = |w - e psi|^2
template <typename T>
__global__ void __launch_bounds__(kThreads) resid_kernel(const T* w, const T* psi, int64_t n, double e,
                                                         double* partials, unsigned int* ticket, double* out) {
  double acc = 0.0;
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads) {
    const double r = double(w[k]) - e * double(psi[k]);
    acc += r * r;
  }
  grid_sum(acc, partials, ticket, out);
}

template <typename T>
__global__ void scale_kernel(T* v, int64_t n, double f) {
  const T c = T(f);
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads)
    v[k] *= c;
}

int vec_grid(int64_t n) {
  const int64_t g = (n + 4 * kThreads - 1) / (4 * kThreads);
  return int(std::max<int64_t>(1, std::min<int64_t>(g, int64_t(device_sms()) * 8)));
}

int ensure_work(mcd_ctx* c, int dtype, int max_iter) {
  LanczosWork& w = c->lw;
  const int64_t n = c->idx.n;
  const size_t es = dtype == MCD_F64 ? 8 : 4;
  const int cap = max_iter + 2;
  const int ctas = std::max<int>(int(c->idx.A.n_items), device_sms() * 8) + 8;
  // keep every Krylov vector when it fits in half of the free memory (no
  // second pass for the Ritz vector); else two rotating slots
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t held = w.V ? size_t(w.nvec) * size_t(w.ld) * (w.dtype == MCD_F64 ? 8 : 4) : 0;
  const bool want_store = c->krylov_store == 0 &&
                          double(max_iter + 1) * double(n) * double(es) <= 0.5 * double(free_b + held);
  const int nvec = want_store ? max_iter + 1 : 2;
  if (w.n == n && w.dtype == dtype && w.scal_cap >= cap && w.max_ctas >= ctas && w.nvec >= nvec &&
      w.stored == want_store)
    return MCD_OK;
  free_lanczos(w);
  // slots start on 16-byte boundaries (the update kernel moves 16-byte vectors)
  const int64_t ld = (n + 3) & ~int64_t(3);
  cudaError_t e = cudaMalloc(&w.W, size_t(n) * es + 64);
  if (e == cudaSuccess) e = cudaMalloc(&w.V, size_t(nvec) * size_t(ld) * es + 64);
  if (e == cudaSuccess && dtype == MCD_F32) e = cudaMalloc(&w.psi64, size_t(n) * 8 + 64);
  if (e == cudaSuccess && dtype == MCD_F32) e = cudaMalloc(&w.w64, size_t(n) * 8 + 64);
  if (e == cudaSuccess) e = cudaMalloc(&w.coef, sizeof(double) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&w.scal, sizeof(double) * (2 * cap + 16));
  if (e == cudaSuccess) e = cudaMalloc(&w.partials, sizeof(double) * ctas);
  if (e == cudaSuccess) e = cudaMalloc(&w.ticket, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(w.ticket, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    free_lanczos(w);
    return cuda_fail(c, e, "Lanczos workspace");
  }
  w.n = n;
  w.ld = ld;
  w.dtype = dtype;
  w.nvec = nvec;
  w.stored = want_store;
  w.scal_cap = cap;
  w.max_ctas = ctas;
  return MCD_OK;
}

template <typename T>
int run(mcd_ctx* c, int max_iter, double tol, uint64_t seed, double* E0_out, T* psi, int* iters_out,
        double* resid_out) {
  LanczosWork& w = c->lw;
  const int64_t n = c->idx.n;
  cudaStream_t s = c->stream;
  const Slots sl{w.scal_cap};
  const int vg = vec_grid(n);
  const uint64_t key = smix(smix(seed + kGamma) ^ 0x4C414E43ull);   // stream "LANC"
  T* V = static_cast<T*>(w.V);
  T* W = static_cast<T*>(w.W);
  const bool fp32 = sizeof(T) == 4;
  // Krylov vector s_j: its own slot when all are stored, else slot j % 2
  auto vec = [&](int j) -> T* { return V + int64_t(w.stored ? j : (j & 1)) * w.ld; };

  auto fresh_start = [&]() -> cudaError_t {
    start_kernel<T><<<vg, kThreads, 0, s>>>(vec(0), n, key, w.partials, w.ticket, w.scal + sl.nrm2(0));
    MCD_LAUNCHED(c);
    return cudaGetLastError();
  };
  // one step: W = H s_it (fused <s_it, W> into slot dot(it)), s_{it+1} from W, s_it, s_{it-1}
  auto step = [&](int it) -> int {
    int st = hv_apply(c, vec(it), W, 1, 1, fp32 ? MCD_F32 : MCD_F64, w.partials, sl.dot(it));
    if (st != MCD_OK) return st;
    timing_begin(c, 2);
    update_kernel<T><<<vg, kThreads, 0, s>>>(W, vec(it), vec(it > 0 ? it - 1 : 0), vec(it + 1), n, it, w.scal,
                                             sl, w.partials, w.ticket);
    MCD_LAUNCHED(c);
    timing_end(c);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "Lanczos update");
  };

  cudaError_t e = fresh_start();
  if (e != cudaSuccess) return cuda_fail(c, e, "Lanczos start");
  std::vector<double> nrm2, dot;
  std::vector<double> a, b, ev;
  double E0 = 0.0, resid = INFINITY;
  int m = 0;          // completed steps
  bool done = false, breakdown = false, bad = false;
  const int chunk = 16;
  while (!done && m < max_iter) {
    const int todo = std::min(chunk, max_iter - m);
    for (int k = 0; k < todo; ++k) {
      int st = step(m + k);
      if (st != MCD_OK) return st;
    }
    m += todo;
    nrm2.resize(m + 1);
    dot.resize(m);
    e = cudaMemcpyAsync(nrm2.data(), w.scal, sizeof(double) * (m + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dot.data(), w.scal + sl.dot(0), sizeof(double) * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Lanczos read-back");
    {
      const int ws = take_wait_errors(c);   // a product whose bounded wait gave up is incomplete
      if (ws != MCD_OK) return ws;
    }
    // coefficients a_n = dot_n / nrm2_n, b_n = sqrt(nrm2_n) (n >= 1)
    a.assign(m, 0.0);
    b.assign(m + 1, 0.0);
    int mm = m;
    for (int k = 0; k < m; ++k) {
      a[k] = dot[k] / nrm2[k];
      if (k > 0) b[k] = std::sqrt(nrm2[k]);
      if (!std::isfinite(a[k]) || !std::isfinite(b[k])) { mm = k; bad = true; break; }
    }
    b[m] = std::sqrt(nrm2[m]);
    // invariant subspace: b_{k+1} negligible against the spectrum scale
    double scale = 0.0;
    for (int k = 0; k < mm; ++k) scale = std::max(scale, std::fabs(a[k]) + b[k] + b[k + 1]);
    for (int k = 0; k < mm; ++k) {
      if (b[k + 1] <= 1e-14 * std::max(1.0, scale) || !std::isfinite(b[k + 1])) {
        if (!std::isfinite(b[k + 1])) bad = true;
        mm = k + 1;
        breakdown = true;
        break;
      }
    }
    if (mm == 0) return fail(c, MCD_E_BREAKDOWN, "Lanczos: non-finite first coefficient");
    ev.assign(mm, 0.0);
    E0 = tridiag_lowest(a.data(), b.data(), mm, ev.data());
    resid = (breakdown ? 0.0 : b[mm]) * std::fabs(ev[mm - 1]);
    m = mm;
    if (breakdown || bad) done = true;
    else if (tol > 0 && resid < tol * std::max(1.0, std::fabs(E0))) done = true;
  }
  c->last_a.assign(a.begin(), a.begin() + m);
  c->last_b.assign(b.begin(), b.begin() + m);
  *E0_out = E0;
  *iters_out = m;
  *resid_out = resid;
  if (bad && !breakdown) return fail(c, MCD_E_BREAKDOWN, "Lanczos: non-finite coefficient");
  int status = MCD_OK;
  if (!done && tol > 0) status = MCD_E_NOT_CONVERGED;
  if (!psi && !fp32 && !c->keep_gs) return status;

  // Ritz vector sum_k ev[k] sig_k s_k (change-of-basis Eq. of App. B), in fp64
  // for the fp32 form (whose E0 is then the fp64 Rayleigh quotient of it)
  std::vector<double> coef(m);
  for (int k = 0; k < m; ++k) coef[k] = ev[k] / std::sqrt(nrm2[k]);
  // (fp32 vectors: double-float sum, the same steps whether the vectors are
  // stored or regenerated, so both give the same bits)
  double* p64 = fp32 ? w.psi64 : reinterpret_cast<double*>(psi);
  if (!p64) {
    // fp64 without a caller's vector (the ground state is only kept): the Ritz
    // vector is formed in the kept copy itself and normalised in place below
    if (!c->gs_psi || c->gs_n != n) {
      if (c->gs_psi) cudaFreeAsync(c->gs_psi, s);
      c->gs_psi = nullptr;
      c->gs_valid = false;
      e = cudaMallocAsync(&c->gs_psi, sizeof(double) * n, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "ground-state copy");
      c->gs_n = n;
    }
    p64 = c->gs_psi;
  }
  std::vector<float2> coef32(fp32 ? m : 0);
  for (size_t k = 0; k < coef32.size(); ++k) coef32[k] = split_coef(coef[k]);
  if (w.stored) {
    e = fp32 ? cudaMemcpyAsync(w.coef, coef32.data(), sizeof(float2) * m, cudaMemcpyHostToDevice, s)
             : cudaMemcpyAsync(w.coef, coef.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Ritz coefficients");
    if (fp32)
      combine32_kernel<<<vg, kThreads, 0, s>>>(p64, reinterpret_cast<const float*>(V), n, w.ld, m,
                                               reinterpret_cast<const float2*>(w.coef));
    else
      combine_kernel<<<vg, kThreads, 0, s>>>(p64, reinterpret_cast<const double*>(V), n, w.ld, m, w.coef);
    MCD_LAUNCHED(c);
  } else {
    e = cudaMemsetAsync(p64, 0, sizeof(double) * n, s);
    if (e == cudaSuccess) e = fresh_start();
    if (e != cudaSuccess) return cuda_fail(c, e, "Ritz vector");
    for (int k = 0; k < m; ++k) {
      if (fp32)
        axpy_df_kernel<<<vg, kThreads, 0, s>>>(reinterpret_cast<float2*>(p64),
                                               reinterpret_cast<const float*>(vec(k)), n, coef32[k].x, coef32[k].y);
      else
        axpy64_kernel<<<vg, kThreads, 0, s>>>(p64, reinterpret_cast<const double*>(vec(k)), n, coef[k]);
      MCD_LAUNCHED(c);
      if (k + 1 < m) {
        int st = step(k);
        if (st != MCD_OK) return st;
      }
    }
    if (fp32) {
      finish_df_kernel<<<vg, kThreads, 0, s>>>(p64, n);
      MCD_LAUNCHED(c);
    }
  }
  // |psi|^2, <psi, H psi>, |H psi - E psi|^2 in fp64
  double* hp64 = fp32 ? w.w64 : reinterpret_cast<double*>(W);
  double nn = 0.0, hh = 0.0, rr = 0.0;
  int st = hv_apply(c, p64, hp64, 1, 1, MCD_F64, nullptr, 0);
  if (st != MCD_OK) return st;
  dot_kernel<double><<<vg, kThreads, 0, s>>>(p64, nullptr, n, w.partials, w.ticket, w.scal + sl.misc(0));
  MCD_LAUNCHED(c);
  dot_kernel<double><<<vg, kThreads, 0, s>>>(p64, hp64, n, w.partials, w.ticket, w.scal + sl.misc(1));
  MCD_LAUNCHED(c);
  e = cudaMemcpyAsync(&nn, w.scal + sl.misc(0), 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hh, w.scal + sl.misc(1), 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Ritz norm");
  const double Eq = hh / nn;
  if (fp32) {
    // fp32 form: E0 = Rayleigh quotient of the Ritz vector with an fp64 H~
    // (variational; error quadratic in the Ritz vector's error)
    E0 = Eq;
    *E0_out = Eq;
  }
  resid_kernel<double><<<vg, kThreads, 0, s>>>(hp64, p64, n, E0, w.partials, w.ticket, w.scal + sl.misc(2));
  MCD_LAUNCHED(c);
  e = cudaMemcpyAsync(&rr, w.scal + sl.misc(2), 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Ritz residual");
  {
    const int ws = take_wait_errors(c);
    if (ws != MCD_OK) return ws;
  }
  *resid_out = std::sqrt(rr / nn);
  // keep the normalised ground state for the Green function
  if (!c->gs_psi || c->gs_n != n) {
    if (c->gs_psi) cudaFreeAsync(c->gs_psi, s);
    c->gs_psi = nullptr;
    e = cudaMallocAsync(&c->gs_psi, sizeof(double) * n, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "ground-state copy");
    c->gs_n = n;
  }
  cast_scale_kernel<double><<<vg, kThreads, 0, s>>>(c->gs_psi, p64, n, 1.0 / std::sqrt(nn));
  MCD_LAUNCHED(c);
  c->gs_E0 = E0;
  c->gs_valid = true;
  if (psi) {
    cast_scale_kernel<T><<<vg, kThreads, 0, s>>>(psi, p64, n, 1.0 / std::sqrt(nn));
    MCD_LAUNCHED(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "Ritz output");
  }
  return status;
}

}  // namespace

void free_lanczos(LanczosWork& w) {
  for (void* p : {w.W, w.V, static_cast<void*>(w.psi64), static_cast<void*>(w.w64), static_cast<void*>(w.coef)})
    if (p) cudaFree(p);
  if (w.scal) cudaFree(w.scal);
  if (w.partials) cudaFree(w.partials);
  if (w.ticket) cudaFree(w.ticket);
  w = LanczosWork();
}

int vec_dot(mcd_ctx* c, const void* a, const void* b, int64_t n, int dtype, double* out) {
  LanczosWork& w = c->lw;
  const int vg = vec_grid(n);
  if (dtype == MCD_F64)
    dot_kernel<double><<<vg, kThreads, 0, c->stream>>>(static_cast<const double*>(a), static_cast<const double*>(b),
                                                       n, w.partials, w.ticket, out);
  else
    dot_kernel<float><<<vg, kThreads, 0, c->stream>>>(static_cast<const float*>(a), static_cast<const float*>(b), n,
                                                      w.partials, w.ticket, out);
  MCD_LAUNCHED(c);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "dot");
}

int lanczos_ground(mcd_ctx* c, int max_iter, double tol, uint64_t seed, int dtype, double* E0, void* psi,
                   int* iters, double* residual) {
  int st = ensure_work(c, dtype, max_iter);
  if (st != MCD_OK) return st;
  if (dtype == MCD_F64) return run<double>(c, max_iter, tol, seed, E0, static_cast<double*>(psi), iters, residual);
  return run<float>(c, max_iter, tol, seed, E0, static_cast<float*>(psi), iters, residual);
}

}  // namespace mcd
