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

// sum of squares of W stored values: fp32 partial then one fp64 add
template <typename T, int W>
__device__ __forceinline__ double sumsq(const T* v) {
  T s = T(0);
#pragma unroll
  for (int i = 0; i < W; ++i) s = v[i] * v[i] + s;
  return double(s);
}

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
                                                          T* s_prev, int64_t n, int step, const double* scal,
                                                          Slots sl, double* partials, unsigned int* ticket) {
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
  double acc = 0.0;
  const int64_t nv = n / W;
  for (int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x; q < nv; q += int64_t(gridDim.x) * kThreads) {
    T a[W], b[W], c[W], o[W];
    ld(w + q * W, a);
    ld(s + q * W, b);
    if (use_prev) ld(s_prev + q * W, c);
#pragma unroll
    for (int i = 0; i < W; ++i) o[i] = use_prev ? (al * a[i] + be * b[i] + ga * c[i]) : (al * a[i] + be * b[i]);
    st(s_prev + q * W, o);
    acc += sumsq<T, W>(o);
  }
  // tail
  if (blockIdx.x == 0) {
    for (int64_t k = nv * W + threadIdx.x; k < n; k += kThreads) {
      T o = al * w[k] + be * s[k];
      if (use_prev) o += ga * s_prev[k];
      s_prev[k] = o;
      acc += double(o) * double(o);
    }
  }
  grid_sum(acc, partials, ticket, const_cast<double*>(scal) + sl.nrm2(step + 1));
}

// psi += coef * s
template <typename T>
__global__ void axpy_kernel(T* psi, const T* s, int64_t n, double coef) {
  const T c = T(coef);
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads)
    psi[k] += c * s[k];
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
  return int(std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8)));
}

int ensure_work(mcd_ctx* c, int dtype, int max_iter) {
  LanczosWork& w = c->lw;
  const int64_t n = c->idx.n;
  const size_t es = dtype == MCD_F64 ? 8 : 4;
  const int cap = max_iter + 2;
  const int ctas = std::max<int>(int(c->idx.A.n_items), 152 * 8) + 8;
  if (w.n == n && w.dtype == dtype && w.scal_cap >= cap && w.max_ctas >= ctas) return MCD_OK;
  free_lanczos(w);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&w.v[i], size_t(n) * es + 64);
  if (e == cudaSuccess) e = cudaMalloc(&w.scal, sizeof(double) * (2 * cap + 16));
  if (e == cudaSuccess) e = cudaMalloc(&w.partials, sizeof(double) * ctas);
  if (e == cudaSuccess) e = cudaMalloc(&w.ticket, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(w.ticket, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    free_lanczos(w);
    return cuda_fail(c, e, "Lanczos workspace");
  }
  w.n = n;
  w.dtype = dtype;
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
  T* buf[3] = {static_cast<T*>(w.v[0]), static_cast<T*>(w.v[1]), static_cast<T*>(w.v[2])};

  auto fresh_start = [&]() -> cudaError_t {
    start_kernel<T><<<vg, kThreads, 0, s>>>(buf[0], n, key, w.partials, w.ticket, w.scal + sl.nrm2(0));
    MCD_LAUNCHED(c);
    return cudaGetLastError();
  };
  // one step: C -> W = H C (dot into slot), P <- s_{n+1}
  auto step = [&](int it, T*& P, T*& C, T* W) -> int {
    int st = hv_apply(c, C, W, 1, 1, sizeof(T) == 8 ? MCD_F64 : MCD_F32, w.partials, sl.dot(it));
    if (st != MCD_OK) return st;
    timing_begin(c, 2);
    update_kernel<T><<<vg, kThreads, 0, s>>>(W, C, P, n, it, w.scal, sl, w.partials, w.ticket);
    MCD_LAUNCHED(c);
    timing_end(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "Lanczos update");
    T* t = P;
    P = C;
    C = t;
    return MCD_OK;
  };

  cudaError_t e = fresh_start();
  if (e != cudaSuccess) return cuda_fail(c, e, "Lanczos start");
  T* P = buf[1];
  T* C = buf[0];
  T* W = buf[2];
  std::vector<double> nrm2, dot;
  std::vector<double> a, b, vec;
  double E0 = 0.0, resid = INFINITY;
  int m = 0;          // completed steps
  bool done = false, breakdown = false, bad = false;
  const int chunk = 16;
  while (!done && m < max_iter) {
    const int todo = std::min(chunk, max_iter - m);
    for (int k = 0; k < todo; ++k) {
      int st = step(m + k, P, C, W);
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
    vec.assign(mm, 0.0);
    E0 = tridiag_lowest(a.data(), b.data(), mm, vec.data());
    resid = (breakdown ? 0.0 : b[mm]) * std::fabs(vec[mm - 1]);
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

  if (psi) {
    // second pass: regenerate s_0..s_{m-1}; psi = sum c_k sig_k s_k
    e = cudaMemsetAsync(psi, 0, sizeof(T) * n, s);
    if (e == cudaSuccess) e = fresh_start();
    if (e != cudaSuccess) return cuda_fail(c, e, "Ritz vector");
    P = buf[1];
    C = buf[0];
    for (int k = 0; k < m; ++k) {
      const double sig = 1.0 / std::sqrt(nrm2[k]);
      axpy_kernel<T><<<vg, kThreads, 0, s>>>(psi, C, n, vec[k] * sig);
      MCD_LAUNCHED(c);
      if (k + 1 < m) {
        int st = step(k, P, C, W);
        if (st != MCD_OK) return st;
      }
    }
    // normalise, then |H psi - E0 psi|
    double nn = 0.0, rr = 0.0;
    dot_kernel<T><<<vg, kThreads, 0, s>>>(psi, nullptr, n, w.partials, w.ticket, w.scal + sl.misc(0));
    MCD_LAUNCHED(c);
    e = cudaMemcpyAsync(&nn, w.scal + sl.misc(0), 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Ritz norm");
    scale_kernel<T><<<vg, kThreads, 0, s>>>(psi, n, 1.0 / std::sqrt(nn));
    MCD_LAUNCHED(c);
    int st = hv_apply(c, psi, W, 1, 1, sizeof(T) == 8 ? MCD_F64 : MCD_F32, nullptr, 0);
    if (st != MCD_OK) return st;
    resid_kernel<T><<<vg, kThreads, 0, s>>>(W, psi, n, E0, w.partials, w.ticket, w.scal + sl.misc(1));
    MCD_LAUNCHED(c);
    e = cudaMemcpyAsync(&rr, w.scal + sl.misc(1), 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Ritz residual");
    *resid_out = std::sqrt(rr);
  }
  return status;
}

}  // namespace

void free_lanczos(LanczosWork& w) {
  for (auto& p : w.v) {
    if (p) cudaFree(p);
    p = nullptr;
  }
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
