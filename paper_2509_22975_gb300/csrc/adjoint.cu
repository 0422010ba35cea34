// Adjoint of the projected Hamiltonian product with respect to its
// parameters (Eq. (1): H = sum t_ij c^dag c + sum eps_i n_i + sum U_i n_up n_dn,
// projected on the truncated basis as in App. B).
//
// H~ is linear in (t, eps, U), so for blocks U, V of ncols columns
//   d <U, H~ V> / d t_ij  = sum over connections through bond (i, j) of
//                           sign * <U[row], V[col]>     (both spins, both directions)
//   d <U, H~ V> / d eps_i = sum_k <U[k], V[k]> (n_i,up(k) + n_i,dn(k))
//   d <U, H~ V> / d U_i   = sum_k <U[k], V[k]> n_i,up(k) n_i,dn(k)
// The adjoint with respect to V is H~ U itself (H~ is symmetric).  With
// U = V = |Omega~> these are the Hellmann-Feynman derivatives of E0.
//
// One thread per state of each ordering walks the bonds in the same order as
// its warp; per-bond contributions are reduced across the warp by shuffles and
// across warps and CTAs in a fixed order (fp64), so results do not depend on
// scheduling.
#include <cmath>
#include <vector>

#include "mcd_internal.h"

namespace mcd {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ int adj_find(const uint32_t* a, int lo, int hi, uint32_t key) {
  int len = hi - lo;
  if (len <= 0) return -1;
  const uint32_t* p = a + lo;
  while (len > 1) {
    const int half = len >> 1;
    if (p[half] <= key) p += half;
    len -= half;
  }
  return (*p == key) ? int(p - a) : -1;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ double row_dot(const T* u, int64_t ru, const T* v, int64_t rv, int ncols, int ld) {
  double s = 0.0;
  for (int c = 0; c < ncols; ++c) s = fma(double(u[ru * ld + c]), double(v[rv * ld + c]), s);
  return s;
}

// outputs per CTA: [n_bonds] bond terms, then (PASS_A) [n] eps terms, [n] U terms
template <typename T, bool PASS_A>
__global__ void __launch_bounds__(kThreads) adjoint_kernel(const Layout L, const HamParams hp, const T* __restrict__ u,
                                                           const T* __restrict__ v, int ncols, int ld, int nout,
                                                           double* partials) {
  extern __shared__ double s_acc[];   // [kWarps][nout]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * nout; i += kThreads) s_acc[i] = 0.0;
  __syncthreads();
  const int n = hp.n_sites;
  const int64_t stride = int64_t(gridDim.x) * kThreads;
  // every thread of the grid runs the same number of rounds (shuffles stay uniform)
  const int64_t rounds = (L.n + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t k = r * stride + int64_t(blockIdx.x) * kThreads + threadIdx.x;
    const bool live = k < L.n;
    int bbase = 0, bend = 0;
    uint32_t m = 0, major = 0;
    int64_t row = 0;
    if (live) {
      int64_t lo = 0, len = L.nblk;
      while (len > 1) {
        const int64_t h = len >> 1;
        if (L.blk_off[lo + h] <= uint32_t(k)) lo += h;
        len -= h;
      }
      bbase = int(L.blk_off[lo]);
      bend = int(L.blk_off[lo + 1]);
      m = L.minor[k];
      major = L.blk_major[lo];
      row = PASS_A ? k : int64_t(L.perm[k]);
    }
    for (int b = 0; b < hp.n_bonds; ++b) {
      double val = 0.0;
      const uint32_t mk = hp.bonds[b].mask;
      if (live && __popc(m & mk) == 1) {
        const int q = adj_find(L.minor, bbase, bend, m ^ mk);
        if (q >= 0) {
          const int64_t col = PASS_A ? int64_t(q) : int64_t(L.perm[q]);
          val = row_dot(u, row, v, col, ncols, ld);
          if (__popc(m & hp.bonds[b].between) & 1) val = -val;
        }
      }
      val = warp_sum(val);
      if (lane == 0) s_acc[warp * nout + b] += val;
    }
    if (PASS_A) {
      // diagonal terms: up word = block major, dn word = minor
      const double d = live ? row_dot(u, row, v, row, ncols, ld) : 0.0;
      for (int i = 0; i < n; ++i) {
        const int nu = live ? int((major >> i) & 1u) : 0, nd = live ? int((m >> i) & 1u) : 0;
        const double e = warp_sum(d * double(nu + nd));
        const double uu = warp_sum(d * double(nu & nd));
        if (lane == 0) {
          s_acc[warp * nout + hp.n_bonds + i] += e;
          s_acc[warp * nout + hp.n_bonds + n + i] += uu;
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nout; i += kThreads) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += s_acc[w * nout + i];
    partials[int64_t(blockIdx.x) * nout + i] = s;
  }
}

__global__ void adjoint_reduce_kernel(const double* partials, int nparts, int nout, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nout) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += partials[int64_t(p) * nout + i];
  out[i] = s;
}

}  // namespace

int hv_adjoint(mcd_ctx* c, const void* u, const void* v, int ncols, int ld, int dtype, double* grad_t,
               double* grad_eps, double* grad_U) {
  const int n = c->n;
  const int nb = c->hp->n_bonds;
  const int nout = nb + 2 * n;
  const int ctas = device_sms() * 4;
  cudaStream_t s = c->stream;
  double *part = nullptr, *out = nullptr;
  cudaError_t e = cudaMallocAsync(&part, sizeof(double) * size_t(ctas) * nout * 2, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&out, sizeof(double) * nout * 2, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(part, s);
    return cuda_fail(c, e, "adjoint buffers");
  }
  const size_t smem = sizeof(double) * kWarps * nout;
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(adjoint_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(adjoint_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(adjoint_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(adjoint_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  }
  if (dtype == MCD_F64) {
    adjoint_kernel<double, false><<<ctas, kThreads, smem, s>>>(c->idx.B, *c->hp, static_cast<const double*>(u),
                                                               static_cast<const double*>(v), ncols, ld, nout, part);
    adjoint_kernel<double, true><<<ctas, kThreads, smem, s>>>(c->idx.A, *c->hp, static_cast<const double*>(u),
                                                              static_cast<const double*>(v), ncols, ld, nout,
                                                              part + size_t(ctas) * nout);
  } else {
    adjoint_kernel<float, false><<<ctas, kThreads, smem, s>>>(c->idx.B, *c->hp, static_cast<const float*>(u),
                                                              static_cast<const float*>(v), ncols, ld, nout, part);
    adjoint_kernel<float, true><<<ctas, kThreads, smem, s>>>(c->idx.A, *c->hp, static_cast<const float*>(u),
                                                             static_cast<const float*>(v), ncols, ld, nout,
                                                             part + size_t(ctas) * nout);
  }
  c->launches += 2;
  adjoint_reduce_kernel<<<(nout + 255) / 256, 256, 0, s>>>(part, ctas, nout, out);
  adjoint_reduce_kernel<<<(nout + 255) / 256, 256, 0, s>>>(part + size_t(ctas) * nout, ctas, nout, out + nout);
  c->launches += 2;
  std::vector<double> h(size_t(nout) * 2);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), out, sizeof(double) * nout * 2, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(part, s);
  cudaFreeAsync(out, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint");
  if (grad_t) {
    for (int i = 0; i < n * n; ++i) grad_t[i] = 0.0;
    for (int b = 0; b < nb; ++b) {
      const uint32_t mk = c->hp->bonds[b].mask;
      const int i = __builtin_ctz(mk), j = 31 - __builtin_clz(mk);
      const double g = h[b] + h[nout + b];   // up-spin hops (B) + down-spin hops (A)
      grad_t[size_t(i) * n + j] = g;
      grad_t[size_t(j) * n + i] = g;
    }
  }
  for (int i = 0; i < n; ++i) {
    if (grad_eps) grad_eps[i] = h[nout + nb + i];
    if (grad_U) grad_U[i] = h[nout + nb + n + i];
  }
  return MCD_OK;
}

}  // namespace mcd
