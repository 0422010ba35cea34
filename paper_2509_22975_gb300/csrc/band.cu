// Band Lanczos Green function (Sec. "Subspace of the Green function",
// Sec. "Further truncation", App. C) on the device.
//
// 1. Target-weight truncation of the ground state (host sort of |c_n|^2).
// 2. Excited bases F~+ = U_mu c^dag_mu F~, F~- = U_mu c_mu F~ (host,
//    sorted unique), each installed in an internal context of the
//    neighbouring sector so that its H~ product runs on the same kernels.
// 3. Start block Phi[:, nu] = c^(dag)_nu |Omega~> (kernel: for every excited
//    state, remove/add the orbital's electron and search the kept ground-state
//    words; the fermionic sign counts the occupied modes before the orbital).
// 4. Band Lanczos in blocked form: W = H~ V_k (blocked H~V kernels, one
//    column per active Krylov vector), A_k = V_k^T W, W -= V_k A_k +
//    V_{k-1} B_k^T, repeated once (classical Gram-Schmidt twice, fp64 Gram
//    matrices), then a rank-revealing Cholesky QR of W (column pivoting;
//    columns whose remaining norm falls below 1e-10 of their norm before
//    orthogonalisation are deflated, as band Lanczos does) gives V_{k+1} and
//    B_{k+1}.  H_eff is block tridiagonal (banded) with blocks A_k, B_k.
// 5. Eigenpairs of H_eff (host), Q = R0^T S[first block], and the Lehmann
//    sums of the Q-matrix Eqs. summed over the particle and hole runs.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "hv_common.cuh"
#include "mcd_internal.h"

namespace mcd {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxOrb = 64;

struct OrbParams {
  int L;
  int dagger;      // 1: start vectors c^dag |Omega>, 0: c |Omega>
  int n_sites;
  int site[kMaxOrb];
  int spin[kMaxOrb];
};

// Phi[x][nu] = <x| c^(dag)_nu |Omega_t>, x in the excited basis.
template <typename T>
__global__ void start_vec_kernel(const uint64_t* __restrict__ exc, int64_t ne, const uint64_t* __restrict__ gw,
                                 const double* __restrict__ gc, int64_t ng, T* phi, int ld, const OrbParams op) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ne) return;
  const uint64_t x = exc[k];
  const int n = op.n_sites;
  const uint64_t half = n == 32 ? 0xFFFFFFFFull : ((1ull << n) - 1);
  for (int nu = 0; nu < op.L; ++nu) {
    const int sh = op.spin[nu] == 0 ? n + op.site[nu] : op.site[nu];
    const uint64_t bit = 1ull << sh;
    double val = 0.0;
    const bool present = (x & bit) != 0;
    if (present == bool(op.dagger)) {
      const uint64_t w = x ^ bit;   // the ground-state word the orbital acts on
      int64_t lo = 0, len = ng;
      while (len > 1) {
        const int64_t h = len >> 1;
        if (gw[lo + h] <= w) lo += h;
        len -= h;
      }
      if (ng > 0 && gw[lo] == w) {
        // occupied modes before the orbital's mode (order: up 0..n-1, dn 0..n-1)
        const uint32_t up = uint32_t(w >> n), dn = uint32_t(w & half);
        const int i = op.site[nu];
        const uint32_t below = (i == 0) ? 0u : (0xFFFFFFFFu >> (32 - i));
        const int before = op.spin[nu] == 0 ? __popc(up & below) : __popc(up) + __popc(dn & below);
        val = (before & 1) ? -gc[lo] : gc[lo];
      }
    }
    phi[k * ld + nu] = T(val);
  }
}

// C[a][b] partial sums over rows of X[:, a] * Y[:, b]; one row of partials per CTA.
template <typename T>
__global__ void __launch_bounds__(kThreads) gram_kernel(const T* __restrict__ X, int pa, const T* __restrict__ Y,
                                                        int pb, int ld, int64_t n, double* partials) {
  constexpr int kRows = 32;
  __shared__ double xs[kRows][kMaxOrb];
  __shared__ double ys[kRows][kMaxOrb];
  const int npair = pa * pb;
  constexpr int kPer = kMaxOrb * kMaxOrb / kThreads;   // 16 pairs per thread at most
  double acc[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) acc[u] = 0.0;
  for (int64_t r0 = int64_t(blockIdx.x) * kRows; r0 < n; r0 += int64_t(gridDim.x) * kRows) {
    for (int e = threadIdx.x; e < kRows * kMaxOrb; e += kThreads) {
      const int rr = e / kMaxOrb, cc = e % kMaxOrb;
      const int64_t r = r0 + rr;
      xs[rr][cc] = (r < n && cc < pa) ? double(X[r * ld + cc]) : 0.0;
      ys[rr][cc] = (r < n && cc < pb) ? double(Y[r * ld + cc]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int pr = threadIdx.x + u * kThreads;
      if (pr < npair) {
        const int ia = pr / pb, ib = pr % pb;
        double s = acc[u];
        for (int rr = 0; rr < kRows; ++rr) s = fma(xs[rr][ia], ys[rr][ib], s);
        acc[u] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int pr = threadIdx.x + u * kThreads;
    if (pr < npair) partials[int64_t(blockIdx.x) * npair + pr] = acc[u];
  }
}

// fp32 vectors: the same partial sums on the tensor cores.  Every value is
// split exactly into three bf16 pieces, x = x0 + x1 + x2 (round to nearest
// leaves at most 16 and then 8 significant bits, so the third piece is the
// exact remainder); the products x_i y_j with i + j <= 2 are exact in fp32
// and the warp-level MMA (m16n8k16, bf16 in, fp32 accumulate) sums them over
// one chunk of rows; each chunk's fp32 sums are then added to a double-float
// (hi, lo) per Gram entry, whose hi + lo goes into the CTA's fp64 partial.
// The dropped products are below 2^-24 of |x y| and the fp32 rounding stays
// inside each chunk, so an entry carries about 2^-24 sqrt(6 n) rms(x y) of
// error: ~1e-11 of |x| |y| on 5e7 rows.
//
// CTA: 8 warps, kGR rows per iteration.  The slices are kept transposed in
// shared memory (orbital-major, two rows per 32-bit word, kGW words per
// orbital, kGW = 4 mod 32, so fragment loads hit 32 distinct banks).  The
// output (pa x pb, padded to 16 x 8 tiles) is cut into warp blocks of 2 x 2
// tiles; with fewer than 8 blocks, the warps of one block split the chunk's
// 16-row steps between them.
constexpr int kGR = 128;                 // rows per CTA iteration
constexpr int kGW = kGR / 2 + 4;         // 32-bit words per orbital and slice

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// four 8x8 bf16 matrices from shared memory; lane L gives the address of row
// L % 8 of matrix L / 8, register j receives matrix j in the MMA fragment layout
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const uint32_t* row) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(row))));
}

// round-to-nearest bf16 of (va, vb) as one word (va in the low half), and
// va, vb minus those values (exact)
__device__ __forceinline__ uint32_t bf16x2_split(float& va, float& vb) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(va, vb);
  const uint32_t w = *reinterpret_cast<const uint32_t*>(&h);
  va = __fsub_rn(va, __uint_as_float(w << 16));
  vb = __fsub_rn(vb, __uint_as_float(w & 0xFFFF0000u));
  return w;
}

// two exact bf16 integers (|q| <= 256) as one word, qa in the low half
__device__ __forceinline__ uint32_t bf16x2_pack(float qa, float qb) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(qa, qb);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void gram_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}

// rows [r0, r0 + kGR) of M (ld floats each, contiguous) into raw, as 16-byte
// copies (the last one may run up to 12 bytes past row n - 1: the blocks are
// allocated with room for it)
__device__ __forceinline__ void gram_fetch(const float* __restrict__ M, int ld, int64_t n, int64_t r0, float* raw) {
  const int64_t rows = (n - r0 < kGR) ? n - r0 : kGR;
  const int units = int((rows * ld * 4 + 15) / 16);
  const unsigned char* src = reinterpret_cast<const unsigned char*>(M + r0 * ld);
  for (int u = threadIdx.x; u < units; u += kThreads)
    gram_cp16(reinterpret_cast<unsigned char*>(raw) + 16 * u, src + 16 * u);
}

// the chunk's columns [0, p) as three transposed bf16 slices: word (s, c, kp)
// holds rows 2 kp (low half) and 2 kp + 1; rows at or past n are zero.  A warp
// takes tiles of 8 columns x 4 row pairs, lane = (column lane / 4, pair lane %
// 4): its stores (bank 4 c + kp, the word stride being 4 mod 32) hit 32 banks.
__device__ __forceinline__ void gram_split(const float* raw, int p, int ld, int64_t rows, uint32_t* sl, int cpad,
                                           int c0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nct = (p + 7) / 8;
  const int cl = lane >> 2, kl = lane & 3;
  for (int tile = warp; tile < nct * (kGR / 8); tile += kThreads / 32) {
    const int kb = tile / nct;
    const int c = (tile - kb * nct) * 8 + cl, kp = kb * 4 + kl;
    if (c >= p) continue;
    float va = 2 * kp < rows ? raw[(2 * kp) * ld + c] : 0.f;
    float vb = 2 * kp + 1 < rows ? raw[(2 * kp + 1) * ld + c] : 0.f;
    sl[(c0 + c) * kGW + kp] = bf16x2_split(va, vb);
    sl[(cpad + c0 + c) * kGW + kp] = bf16x2_split(va, vb);
    sl[(2 * cpad + c0 + c) * kGW + kp] = bf16x2_pack(va, vb);   // the exact remainder
  }
}

// shared memory of gram_tc_kernel (words): raw rows of X1, X2 (if any) and
// Y (unless Y is X1), then the slices of X = [X1 X2] and (unless Y is X1) of Y
struct GramSmem {
  int Mp, Np, kparts, raw_words, xs_words, ys_words;
  bool same;
  __host__ __device__ GramSmem(int pa, int pb, int ld, bool same_, bool two) {
    same = same_;
    Mp = (pa + 15) / 16 * 16;
    Np = (pb + 7) / 8 * 8;
    const int nblk = ((Mp / 16 + 1) / 2) * ((Np / 8 + 1) / 2);
    kparts = nblk >= 5 ? 1 : (nblk >= 3 ? 2 : (nblk == 2 ? 4 : 8));
    raw_words = (1 + (two ? 1 : 0) + (same ? 0 : 1)) * kGR * ld;
    xs_words = 3 * Mp * kGW;
    ys_words = same ? 0 : 3 * Np * kGW;
  }
  __host__ __device__ size_t bytes() const {
    const size_t main = size_t(raw_words + xs_words + ys_words) * 4;
    const size_t red = size_t(kparts) * Mp * Np * 8;
    return main > red ? main : red;
  }
};

// G = [X1 X2]^T Y (pa = pa1 + pa2 rows: X1's columns, then X2's; X2 may be
// null with pa2 = 0); Y = X1 with pb = pa1 shares X1's slices.
__global__ void __launch_bounds__(kThreads, 2) gram_tc_kernel(const float* __restrict__ X1, int pa1,
                                                              const float* __restrict__ X2, int pa2,
                                                              const float* __restrict__ Y, int pb, int ld, int64_t n,
                                                              double* partials) {
  extern __shared__ __align__(16) uint32_t s_gram[];
  const int pa = pa1 + pa2;
  const bool two = pa2 > 0;
  const GramSmem L(pa, pb, ld, Y == X1 && pb == pa1, two);
  const int Mt = L.Mp / 16, Nt = L.Np / 8, Mp = L.Mp;
  float* raw_x = reinterpret_cast<float*>(s_gram);
  float* raw_x2 = raw_x + kGR * ld;
  float* raw_y = L.same ? raw_x : raw_x + (two ? 2 : 1) * kGR * ld;
  uint32_t* xs = s_gram + L.raw_words;                           // [3][Mp][kGW]
  uint32_t* ys = L.same ? xs : xs + L.xs_words;                  // [3][yst][kGW]
  const int yst = L.same ? Mp : L.Np;
  for (int i = threadIdx.x; i < L.xs_words + L.ys_words; i += kThreads) xs[i] = 0u;   // padding stays zero
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int nnb = (Nt + 1) / 2, nblk = ((Mt + 1) / 2) * nnb;
  const int kparts = L.kparts;
  const bool busy = warp < nblk * kparts;
  const int blk = warp % nblk, kp = warp / nblk;
  const int mt0 = (blk / nnb) * 2, nt0 = (blk % nnb) * 2;
  constexpr int kSteps = kGR / 16;
  const int ksteps = kSteps / kparts, ks0 = kp * ksteps;
  float acc[2][2][4], dh[2][2][4], dl[2][2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = dh[i][j][q] = dl[i][j][q] = 0.f;
  const int64_t step = int64_t(gridDim.x) * kGR;
  int64_t r0 = int64_t(blockIdx.x) * kGR;
  if (r0 < n) {
    gram_fetch(X1, ld, n, r0, raw_x);
    if (two) gram_fetch(X2, ld, n, r0, raw_x2);
    if (!L.same) gram_fetch(Y, ld, n, r0, raw_y);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (; r0 < n; r0 += step) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();   // the chunk's rows have landed; the previous chunk's slices are consumed
    const int64_t rows = (n - r0 < kGR) ? n - r0 : kGR;
    gram_split(raw_x, pa1, ld, rows, xs, Mp, 0);
    if (two) gram_split(raw_x2, pa2, ld, rows, xs, Mp, pa1);
    if (!L.same) gram_split(raw_y, pb, ld, rows, ys, yst, 0);
    __syncthreads();   // slices ready, raw rows free: the next chunk loads during the products
    if (r0 + step < n) {
      gram_fetch(X1, ld, n, r0 + step, raw_x);
      if (two) gram_fetch(X2, ld, n, r0 + step, raw_x2);
      if (!L.same) gram_fetch(Y, ld, n, r0 + step, raw_y);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (!busy) continue;
    // fragment rows of this lane for ldmatrix: A (row-major m x k) matrices
    // (m lo, k lo), (m hi, k lo), (m lo, k hi), (m hi, k hi); B (n x k) matrices
    // (n tile 0, k lo), (n tile 0, k hi), (n tile 1, k lo), (n tile 1, k hi).
    // Rows of tiles past the matrix are clamped to its last row (their products
    // are not formed).
    const int lr = lane & 7, lm = lane >> 3;
    int arow[2], brow;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) arow[mi] = min((mt0 + mi) * 16 + lr + (lm & 1) * 8, Mp - 1);
    brow = min(nt0 * 8 + (lm >> 1) * 8 + lr, Nt * 8 - 1);
    const int akoff = (lm >> 1) * 4, bkoff = (lm & 1) * 4;   // words of the k hi half
    for (int ks = ks0; ks < ks0 + ksteps; ++ks) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        uint32_t a[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) ldmatrix_x4(a[mi], xs + (i * Mp + arow[mi]) * kGW + ks * 8 + akoff);
#pragma unroll
        for (int j = 0; i + j < 3; ++j) {
          uint32_t b[4];
          ldmatrix_x4(b, ys + (j * yst + brow) * kGW + ks * 8 + bkoff);
          const uint32_t b0[2] = {b[0], b[1]}, b1[2] = {b[2], b[3]};
#pragma unroll
          for (int mi = 0; mi < 2; ++mi) {
            if (mt0 + mi >= Mt) continue;
            mma_bf16_16816(acc[mi][0], a[mi], b0);
            if (nt0 + 1 < Nt) mma_bf16_16816(acc[mi][1], a[mi], b1);
          }
        }
      }
    }
    // the chunk's sums into the double-float accumulators
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          df_add(dh[mi][ni][q], dl[mi][ni][q], acc[mi][ni][q]);
          acc[mi][ni][q] = 0.f;
        }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  // CTA partial: the warps' entries (fp64) by split, summed in split order
  __syncthreads();
  double* red = reinterpret_cast<double*>(s_gram);   // [kparts][Mp][Np]
  const int Np = L.Np;
  if (busy) {
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
        if (mt0 + mi < Mt && nt0 + ni < Nt) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int m = (mt0 + mi) * 16 + g + (q >> 1) * 8;
            const int nn = (nt0 + ni) * 8 + 2 * t + (q & 1);
            red[(int64_t(kp) * Mp + m) * Np + nn] = double(dh[mi][ni][q]) + double(dl[mi][ni][q]);
          }
        }
  }
  __syncthreads();
  const int npair = pa * pb;
  for (int pr = threadIdx.x; pr < npair; pr += kThreads) {
    const int ia = pr / pb, ib = pr - ia * pb;
    double v = 0.0;
    for (int k = 0; k < kparts; ++k) v += red[(int64_t(k) * Mp + ia) * Np + ib];
    partials[int64_t(blockIdx.x) * npair + pr] = v;
  }
}

__global__ void reduce_partials_kernel(const double* partials, int nparts, int npair, double* out) {
  const int pr = blockIdx.x * blockDim.x + threadIdx.x;
  if (pr >= npair) return;
  double s = 0.0;
  for (int i = 0; i < nparts; ++i) s += partials[int64_t(i) * npair + pr];
  out[pr] = s;
}

// (hi, lo) += x (ch + cl) in double-float: the product x ch split exactly by
// an FMA, x cl added to its error term, then Knuth's two-sum
__device__ __forceinline__ void df_add(float& hi, float& lo, float x, float ch, float cl) {
  const float p = x * ch;
  const float e = fmaf(x, ch, -p) + x * cl;
  const float sum = hi + p, bb = sum - hi;
  lo += ((hi - (sum - bb)) + (p - bb)) + e;
  hi = sum;
}


// fp32 vectors, K = p1 + p2 <= 64 and pw <= 32: the same combination on the
// tensor cores with exact integer sums.  Each row r of [X1 X2] is scaled by a
// power of two 2^(8 - e_r) (its largest |x| < 2^e_r) and cut into four
// round-to-nearest slices of at most 8 bits (|q_0| <= 256, |q_i| <= 128: bf16
// integers), the coefficients likewise per column j (scale 2^(8 - f_j), cut on
// the host from the fp64 values).  The MMA sums the slice products of one
// level l = i + j (i, j < 4, l <= 3) into an fp32 accumulator of its own:
// integers below 4 * 64 * 2^15 < 2^24, so every sum is exact.  The four levels
// are then combined in double-float, scaled by 2^(e_r + f_j - 16), beta W is
// added exactly and the result rounded once to fp32.  What is lost are the
// slices' remainders, below 2^-33 of the row's and the column's largest
// entries: ~1e-9 of sum |x c|.
constexpr int kCK = 64;          // largest K of the tensor-core combination
constexpr int kCN = 32;          // largest pw
constexpr int kCW = kCK / 2 + 4; // 32-bit words per coefficient column and slice (= 4 mod 32)

// this thread's values of rows r0 + g, r0 + g + 8 and columns 16 ks + 2t + {0, 1, 8, 9} of [X1 X2]
template <int KS>
__device__ __forceinline__ void combine_tc_load(const float* __restrict__ X1, int p1, const float* __restrict__ X2,
                                                int K, int ld, int64_t n, int64_t r0, int g, int t,
                                                float (&v)[2][KS][4]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t r = r0 + g + 8 * h;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 16 * ks + 2 * t + (q & 1) + (q >> 1) * 8;
        float x = 0.f;
        if (r < n && k < K) x = k < p1 ? __ldg(X1 + r * ld + k) : __ldg(X2 + r * ld + (k - p1));
        v[h][ks][q] = x;
      }
  }
}

template <int KS, int NT>
__global__ void __launch_bounds__(kThreads, 2) block_combine_tc_kernel(const float* W, float* out, int pw, float bh,
                                                                       float bl, const float* __restrict__ X1, int p1,
                                                                       const float* __restrict__ X2, int p2,
                                                                       const uint32_t* __restrict__ cslices,
                                                                       const int* __restrict__ fexp, int ld,
                                                                       int64_t n) {
  __shared__ uint32_t s_c[4 * NT * 8 * kCW];   // [slice][n][word of k pairs]
  __shared__ int s_f[NT * 8];
  for (int i = threadIdx.x; i < 4 * NT * 8 * kCW; i += kThreads) s_c[i] = cslices[i];
  for (int i = threadIdx.x; i < NT * 8; i += kThreads) s_f[i] = fexp[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int K = p1 + p2;
  const int64_t ntile = (n + 15) / 16;
  const int64_t stride = int64_t(gridDim.x) * (kThreads / 32);
  int64_t tile = int64_t(blockIdx.x) * (kThreads / 32) + warp;
  float v[2][KS][4];
  if (tile < ntile) combine_tc_load<KS>(X1, p1, X2, K, ld, n, tile * 16, g, t, v);
  for (; tile < ntile; tile += stride) {
    const int64_t r0 = tile * 16;
    // row scales: the largest |x| of the row (over the quad's four threads)
    int er[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float mx = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int q = 0; q < 4; ++q) mx = fmaxf(mx, fabsf(v[h][ks][q]));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      // mx in [2^(e-1), 2^e); rows below 2^-119 are taken as zero
      const int e = int((__float_as_uint(mx) >> 23) & 0xFFu) - 126;
      const bool live = mx >= 0x1p-119f;
      er[h] = live ? e : 0;
      const float sc = live ? __uint_as_float(uint32_t(127 + 8 - e) << 23) : 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks)
#pragma unroll
        for (int q = 0; q < 4; ++q) v[h][ks][q] *= sc;   // exact: |v| < 256
    }
    // the four slices as A fragments (q = rint(v), v <- 256 (v - q), both exact)
    uint32_t a[4][KS][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        float qi[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            qi[h][q] = rintf(v[h][ks][q]);
            v[h][ks][q] = __fmul_rn(__fsub_rn(v[h][ks][q], qi[h][q]), 256.f);
          }
        a[i][ks][0] = bf16x2_pack(qi[0][0], qi[0][1]);
        a[i][ks][1] = bf16x2_pack(qi[1][0], qi[1][1]);
        a[i][ks][2] = bf16x2_pack(qi[0][2], qi[0][3]);
        a[i][ks][3] = bf16x2_pack(qi[1][2], qi[1][3]);
      }
    // the next tile's values load while this one is multiplied
    if (tile + stride < ntile) combine_tc_load<KS>(X1, p1, X2, K, ld, n, (tile + stride) * 16, g, t, v);
    // one 8-column tile at a time: the MMA sums the slice products with
    // i + j = l into the level-l accumulator (exact fp32 integers); the
    // levels then go into a double-float with weight 2^(-8 l)
#pragma unroll 1
    for (int nt = 0; nt < NT; ++nt) {
      float acc[4][4];
#pragma unroll
      for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[l][q] = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; i + j < 4; ++j)
#pragma unroll
          for (int ks = 0; ks < KS; ++ks) {
            const uint32_t* bp = s_c + (j * NT * 8 + nt * 8 + g) * kCW + ks * 8 + t;
            const uint32_t b[2] = {bp[0], bp[4]};
            mma_bf16_16816(acc[i + j], a[i][ks], b);
          }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int h = q >> 1;
        const int64_t r = r0 + g + 8 * h;
        const int j = nt * 8 + 2 * t + (q & 1);
        if (r >= n || j >= pw) continue;
        float oh = acc[0][q], ol = 0.f;
        df_add(oh, ol, __fmul_rn(acc[1][q], 0x1p-8f));
        df_add(oh, ol, __fmul_rn(acc[2][q], 0x1p-16f));
        df_add(oh, ol, __fmul_rn(acc[3][q], 0x1p-24f));
        const int sh = er[h] + s_f[j] - 16;
        float hi, lo;
        if (sh >= -126 && sh <= 127) {   // a power of two: exact
          const float f = __uint_as_float(uint32_t(127 + sh) << 23);
          hi = oh * f;
          lo = ol * f;
        } else {
          hi = ldexpf(oh, sh);
          lo = ldexpf(ol, sh);
        }
        if (bh != 0.f || bl != 0.f) df_add(hi, lo, W[r * ld + j], bh, bl);
        out[r * ld + j] = hi + lo;
      }
    }
  }
}

// W[r][j] = beta * W[r][j] + sum_i X1[r][i] C1[i][j] + sum_i X2[r][i] C2[i][j]
// (C row-major [p_i][pw], fp64); out may alias W.
template <typename T>
__global__ void block_combine_kernel(const T* W, T* out, int pw, double beta, const T* X1, int p1,
                                     const double* C1, const T* X2, int p2, const double* C2, int ld, int64_t n) {
  const double* __restrict__ c1 = C1;
  const double* __restrict__ c2 = C2;
  const int64_t total = n * pw;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / pw;
    const int j = int(e - r * pw);
    double s = beta == 0.0 ? 0.0 : beta * double(W[r * ld + j]);
    for (int i = 0; i < p1; ++i) s = fma(double(X1[r * ld + i]), __ldg(c1 + i * pw + j), s);
    for (int i = 0; i < p2; ++i) s = fma(double(X2[r * ld + i]), __ldg(c2 + i * pw + j), s);
    out[r * ld + j] = T(s);
  }
}

int grid_for(int64_t work) {
  const int64_t g = (work + kThreads - 1) / kThreads;
  return int(std::max<int64_t>(1, std::min<int64_t>(g, int64_t(device_sms()) * 16)));
}

// Pivoted Cholesky of the p x p Gram G (row-major): G[piv, piv] = R^T R with
// R upper triangular rank x p in pivoted column order.  Columns whose
// remaining norm falls below dtol * ref[j] (norm before orthogonalisation)
// are deflated.  Returns rank; piv[0..p) the column order.
int pivoted_cholesky(int p, const std::vector<double>& G, const std::vector<double>& ref, double dtol,
                     std::vector<int>& piv, std::vector<double>& R) {
  std::vector<double> A = G;
  piv.resize(p);
  for (int i = 0; i < p; ++i) piv[i] = i;
  R.assign(size_t(p) * p, 0.0);
  int rank = 0;
  for (int k = 0; k < p; ++k) {
    // remaining diagonal of the Schur complement
    // pivot: the column with the largest remaining norm relative to its norm
    // before orthogonalisation; deflate the rest when that ratio is <= dtol
    int best = -1;
    double bestv = -1.0, bestrel = -1.0;
    for (int j = k; j < p; ++j) {
      const int c = piv[j];
      double d = A[size_t(c) * p + c];
      for (int i = 0; i < k; ++i) d -= R[size_t(i) * p + j] * R[size_t(i) * p + j];
      const double rel = d / std::max(ref[c] * ref[c], 1e-300);
      if (rel > bestrel) { bestrel = rel; bestv = d; best = j; }
    }
    if (best < 0 || bestv <= 0.0 || std::sqrt(std::max(bestrel, 0.0)) <= dtol) break;
    // swap pivot into position k (also the R columns computed so far)
    std::swap(piv[k], piv[best]);
    for (int i = 0; i < k; ++i) std::swap(R[size_t(i) * p + k], R[size_t(i) * p + best]);
    const double rkk = std::sqrt(bestv);
    R[size_t(k) * p + k] = rkk;
    for (int j = k + 1; j < p; ++j) {
      double s = A[size_t(piv[k]) * p + piv[j]];
      for (int i = 0; i < k; ++i) s -= R[size_t(i) * p + k] * R[size_t(i) * p + j];
      R[size_t(k) * p + j] = s / rkk;
    }
    rank = k + 1;
  }
  return rank;
}

// M (p x r, row-major) with W * M = orthonormal block, from the pivoted
// factor: M = P[:, :r] * inv(R11); and F (r x p) = R P^T so W ~ V F.
void factors(int p, int r, const std::vector<int>& piv, const std::vector<double>& R, std::vector<double>& M,
             std::vector<double>& F) {
  // inverse of the r x r upper-triangular R11 (column order = pivot order)
  std::vector<double> inv(size_t(r) * r, 0.0);
  for (int j = 0; j < r; ++j) {
    inv[size_t(j) * r + j] = 1.0 / R[size_t(j) * p + j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += R[size_t(i) * p + k] * inv[size_t(k) * r + j];
      inv[size_t(i) * r + j] = -s / R[size_t(i) * p + i];
    }
  }
  M.assign(size_t(p) * r, 0.0);
  for (int a = 0; a < r; ++a)
    for (int j = 0; j < r; ++j) M[size_t(piv[a]) * r + j] = inv[size_t(a) * r + j];
  F.assign(size_t(r) * p, 0.0);
  for (int i = 0; i < r; ++i)
    for (int b = 0; b < p; ++b) F[size_t(i) * p + piv[b]] = R[size_t(i) * p + b];
}

struct BandRun {
  std::vector<double> E;   // eigenvalues of H_eff (when the blocks are kept)
  std::vector<double> Q;   // [L][K]                (when the blocks are kept)
  std::vector<double> S;   // [K][K] eigenvectors of H_eff (when the blocks are kept)
  // the block tridiagonal H_eff itself: A_k (p_k x p_k), B_{k+1} (p_{k+1} x p_k),
  // and R0 (p_0 x L) with the start block = V_0 R0
  std::vector<std::vector<double>> A, B;
  std::vector<int> ps;
  std::vector<double> R0;
  int64_t dim = 0;
  int K = 0;
};

// In-place inverse of the p x p complex matrix M (row-major), Gauss-Jordan
// with partial pivoting; false when a pivot vanishes.
bool cinv(int p, std::vector<std::complex<double>>& M) {
  std::vector<int> perm(p);
  for (int i = 0; i < p; ++i) perm[i] = i;
  for (int k = 0; k < p; ++k) {
    int best = k;
    double bv = std::abs(M[size_t(k) * p + k]);
    for (int i = k + 1; i < p; ++i)
      if (std::abs(M[size_t(i) * p + k]) > bv) { bv = std::abs(M[size_t(i) * p + k]); best = i; }
    if (!(bv > 0.0)) return false;
    if (best != k) {
      for (int j = 0; j < p; ++j) std::swap(M[size_t(k) * p + j], M[size_t(best) * p + j]);
      std::swap(perm[k], perm[best]);
    }
    const std::complex<double> inv = 1.0 / M[size_t(k) * p + k];
    M[size_t(k) * p + k] = 1.0;
    for (int j = 0; j < p; ++j) M[size_t(k) * p + j] *= inv;
    for (int i = 0; i < p; ++i) {
      if (i == k) continue;
      const std::complex<double> f = M[size_t(i) * p + k];
      if (f == 0.0) continue;
      M[size_t(i) * p + k] = 0.0;
      for (int j = 0; j < p; ++j) M[size_t(i) * p + j] -= f * M[size_t(k) * p + j];
    }
  }
  // undo the row interchanges as column interchanges of the inverse
  std::vector<std::complex<double>> out(size_t(p) * p);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) out[size_t(i) * p + perm[j]] = M[size_t(i) * p + j];
  M.swap(out);
  return true;
}

// G[z][a][b] += sgn R0[:, a]^T [(w I - H_eff)^{-1}]_{00} R0[:, b] with
// w = z + E0 (particle run, sgn = +1) or w = -z + E0 (hole run, sgn = -1): the
// Lehmann sums of App. C over the eigenpairs of H_eff, evaluated without the
// eigenpairs as the block continued fraction of the block tridiagonal H_eff
// (Schur complements from the last block up: S_k = w - A_k - B_{k+1}^T
// S_{k+1}^{-1} B_{k+1}, then S_0^{-1} is the (0, 0) block of the resolvent).
bool band_resolvent(const BandRun& R, int L, double E0, bool particle, const double* z_re, const double* z_im,
                    int nz, double* G_re, double* G_im) {
  using cd = std::complex<double>;
  const int nb = int(R.A.size());
  if (nb == 0) return true;
  const int p0 = R.ps[0];
  std::vector<cd> S, T, Sn;
  for (int iz = 0; iz < nz; ++iz) {
    const cd z(z_re[iz], z_im[iz]);
    const cd w = particle ? z + E0 : -z + E0;
    const double sgn = particle ? 1.0 : -1.0;
    int p = R.ps[nb - 1];
    S.assign(size_t(p) * p, 0.0);
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) S[size_t(i) * p + j] = (i == j ? w : cd(0.0)) - R.A[nb - 1][size_t(i) * p + j];
    for (int k = nb - 2; k >= 0; --k) {
      if (!cinv(p, S)) return false;             // S_{k+1}^{-1}
      const int q = R.ps[k];                      // B_{k+1}: p x q
      const std::vector<double>& B = R.B[k];
      T.assign(size_t(p) * q, 0.0);               // S^{-1} B
      for (int i = 0; i < p; ++i)
        for (int l = 0; l < p; ++l) {
          const cd sv = S[size_t(i) * p + l];
          if (sv == 0.0) continue;
          for (int j = 0; j < q; ++j) T[size_t(i) * q + j] += sv * B[size_t(l) * q + j];
        }
      Sn.assign(size_t(q) * q, 0.0);
      for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
          cd acc = (i == j ? w : cd(0.0)) - R.A[k][size_t(i) * q + j];
          for (int l = 0; l < p; ++l) acc -= B[size_t(l) * q + i] * T[size_t(l) * q + j];
          Sn[size_t(i) * q + j] = acc;
        }
      S.swap(Sn);
      p = q;
    }
    if (!cinv(p0, S)) return false;
    for (int a = 0; a < L; ++a)
      for (int b = 0; b < L; ++b) {
        cd acc = 0.0;
        for (int i = 0; i < p0; ++i) {
          const double ra = R.R0[size_t(i) * L + a];
          if (ra == 0.0) continue;
          for (int j = 0; j < p0; ++j) acc += ra * S[size_t(i) * p0 + j] * R.R0[size_t(j) * L + b];
        }
        G_re[(size_t(iz) * L + a) * L + b] += sgn * acc.real();
        G_im[(size_t(iz) * L + a) * L + b] += sgn * acc.imag();
      }
  }
  return true;
}

// dst[r][off + j] = src[r][j] (j < p): one Krylov block into the kept [n][kmax] array
template <typename T>
__global__ void keep_block_kernel(const T* src, int ld_src, int p, double* dst, int kmax, int off, int64_t n) {
  const int64_t total = n * p;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / p;
    const int j = int(e - r * p);
    dst[r * kmax + off + j] = double(src[r * ld_src + j]);
  }
}

template <typename T>
class BandLanczos {
 public:
  BandLanczos(mcd_ctx* sub, int L) : c_(sub), L_(L), n_(sub->idx.n) {}
  ~BandLanczos() {
    for (void* p : {static_cast<void*>(B_[0]), static_cast<void*>(B_[1]), static_cast<void*>(B_[2]),
                    static_cast<void*>(part_), static_cast<void*>(gram_), static_cast<void*>(coef_)})
      if (p) cudaFreeAsync(p, c_->stream);
  }

  int alloc() {
    cudaError_t e = cudaSuccess;
    cudaStream_t s = c_->stream;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
      e = cudaMallocAsync(reinterpret_cast<void**>(&B_[i]), size_t(n_) * L_ * sizeof(T) + 64, s);
    nparts_ = grid_for(n_ / 32 + 1);
    if (e == cudaSuccess)
      e = cudaMallocAsync(reinterpret_cast<void**>(&part_), sizeof(double) * size_t(nparts_) * kMaxOrb * kMaxOrb, s);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&gram_), sizeof(double) * kMaxOrb * kMaxOrb, s);
    if (e == cudaSuccess)
      e = cudaMallocAsync(reinterpret_cast<void**>(&coef_), sizeof(double) * 2 * kMaxOrb * kMaxOrb, s);
    if (e != cudaSuccess) return cuda_fail(c_, e, "band Lanczos buffers");
    return MCD_OK;
  }
  T* buf(int i) { return B_[i]; }
  // keep every Krylov block in vall[n][kmax] (fp64) and return all eigenvectors
  void keep_blocks(double* vall, int kmax) {
    vall_ = vall;
    kmax_ = kmax;
  }

  // host G = X[:, :pa]^T Y[:, :pb]
  int gram(const T* X, int pa, const T* Y, int pb, std::vector<double>& G) {
    return gram2(X, pa, nullptr, 0, Y, pb, G);
  }

  // host G = [X1[:, :pa1] X2[:, :pa2]]^T Y[:, :pb] ((pa1 + pa2) x pb, X1's
  // rows first): one pass over the rows in fp32 (pa1 + pa2 <= 2 kMaxSites =
  // 64), one product at a time in fp64
  int gram2(const T* X1, int pa1, const T* X2, int pa2, const T* Y, int pb, std::vector<double>& G) {
    cudaStream_t s = c_->stream;
    const int pa = pa1 + pa2;
    int npair = pa * pb;
    if constexpr (sizeof(T) == 4) {
      if (pa > kMaxOrb) return fail(c_, MCD_E_INVALID, "band Lanczos: Gram of more than 64 columns");
      const size_t smem = GramSmem(pa, pb, L_, Y == X1 && pb == pa1, pa2 > 0).bytes();
      if (smem > 48 * 1024) {
        const cudaError_t ea =
            cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (ea != cudaSuccess) return cuda_fail(c_, ea, "Gram kernel shared memory");
      }
      gram_tc_kernel<<<nparts_, kThreads, smem, s>>>(X1, pa1, pa2 ? X2 : nullptr, pa2, Y, pb, L_, n_, part_);
    } else {
      if (pa2) {   // X2's rows after X1's
        std::vector<double> G1, G2;
        int st = gram2(X1, pa1, nullptr, 0, Y, pb, G1);
        if (st == MCD_OK) st = gram2(X2, pa2, nullptr, 0, Y, pb, G2);
        if (st != MCD_OK) return st;
        G = G1;
        G.insert(G.end(), G2.begin(), G2.end());
        return MCD_OK;
      }
      gram_kernel<T><<<nparts_, kThreads, 0, s>>>(X1, pa1, Y, pb, L_, n_, part_);
    }
    MCD_LAUNCHED(c_);
    reduce_partials_kernel<<<(npair + 255) / 256, 256, 0, s>>>(part_, nparts_, npair, gram_);
    MCD_LAUNCHED(c_);
    G.resize(size_t(npair));
    cudaError_t e = cudaMemcpyAsync(G.data(), gram_, sizeof(double) * npair, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MCD_OK : cuda_fail(c_, e, "Gram");
  }

  // out = beta W + X1 C1 + X2 C2 (C1: p1 x pw, C2: p2 x pw)
  int combine(const T* W, T* out, int pw, double beta, const T* X1, int p1, const std::vector<double>& C1,
              const T* X2, int p2, const std::vector<double>& C2) {
    cudaStream_t s = c_->stream;
    std::vector<double> buf(2 * size_t(kMaxOrb) * kMaxOrb, 0.0);
    std::copy(C1.begin(), C1.begin() + size_t(p1) * pw, buf.begin());
    if (p2) std::copy(C2.begin(), C2.begin() + size_t(p2) * pw, buf.begin() + size_t(kMaxOrb) * kMaxOrb);
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
      const size_t m = size_t(kMaxOrb) * kMaxOrb;
      const float bh = float(beta), bl = float(beta - double(bh));
      const int K = p1 + p2;
      // orbitals share one spin, so a block has at most kMaxSites = 32 columns:
      // K <= 64 and pw <= 32 always hold
      if (K > kCK || pw > kCN) return fail(c_, MCD_E_INVALID, "band Lanczos: block wider than 32 columns");
      // integer slices of the coefficients of [C1; C2] per column (see block_combine_tc_kernel)
      const int KS = (K + 15) / 16, NT = (pw + 7) / 8;
      std::vector<uint16_t> sl(size_t(4) * NT * 8 * kCW * 2, 0);
      std::vector<int> fe(size_t(NT) * 8, 0);
      for (int j = 0; j < pw; ++j) {
        double mx = 0.0;
        for (int k = 0; k < K; ++k)
          mx = std::max(mx, std::fabs(k < p1 ? buf[size_t(k) * pw + j] : buf[m + size_t(k - p1) * pw + j]));
        if (!(mx >= 0x1p-119)) continue;   // a zero column (or one below 2^-119): slices stay zero
        int ex = 0;
        std::frexp(mx, &ex);                // mx in [2^(ex-1), 2^ex)
        fe[j] = ex;
        for (int k = 0; k < K; ++k) {
          double v = std::ldexp(k < p1 ? buf[size_t(k) * pw + j] : buf[m + size_t(k - p1) * pw + j], 8 - ex);
          for (int i = 0; i < 4; ++i) {
            const double qi = std::nearbyint(v);
            v = (v - qi) * 256.0;
            // |qi| <= 256: exact in bf16 (sign, exponent, 7 stored bits)
            const float fq = float(qi);
            uint32_t bits;
            std::memcpy(&bits, &fq, 4);
            sl[(size_t(i) * NT * 8 + j) * kCW * 2 + k] = uint16_t(bits >> 16);
          }
        }
      }
      uint32_t* dsl = reinterpret_cast<uint32_t*>(coef_);
      int* dfe = reinterpret_cast<int*>(dsl + size_t(4) * NT * 8 * kCW);
      e = cudaMemcpyAsync(dsl, sl.data(), sl.size() * 2, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dfe, fe.data(), fe.size() * 4, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(c_, e, "block coefficients");
      const int grid = int(std::max<int64_t>(1, std::min<int64_t>((n_ + 127) / 128, int64_t(device_sms()) * 8)));
      const float* x2 = X2 ? X2 : X1;
#define MCD_COMBINE_TC(ks, nt)                                                                              \
  block_combine_tc_kernel<ks, nt><<<grid, kThreads, 0, s>>>(W, out, pw, bh, bl, X1, p1, x2, p2, dsl, dfe, L_, n_)
      switch (KS * 8 + NT) {
        case 9: MCD_COMBINE_TC(1, 1); break;
        case 10: MCD_COMBINE_TC(1, 2); break;
        case 11: MCD_COMBINE_TC(1, 3); break;
        case 12: MCD_COMBINE_TC(1, 4); break;
        case 17: MCD_COMBINE_TC(2, 1); break;
        case 18: MCD_COMBINE_TC(2, 2); break;
        case 19: MCD_COMBINE_TC(2, 3); break;
        case 20: MCD_COMBINE_TC(2, 4); break;
        case 25: MCD_COMBINE_TC(3, 1); break;
        case 26: MCD_COMBINE_TC(3, 2); break;
        case 27: MCD_COMBINE_TC(3, 3); break;
        case 28: MCD_COMBINE_TC(3, 4); break;
        case 33: MCD_COMBINE_TC(4, 1); break;
        case 34: MCD_COMBINE_TC(4, 2); break;
        case 35: MCD_COMBINE_TC(4, 3); break;
        default: MCD_COMBINE_TC(4, 4); break;
      }
#undef MCD_COMBINE_TC
    } else {
      e = cudaMemcpyAsync(coef_, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return cuda_fail(c_, e, "block coefficients");
      block_combine_kernel<T><<<grid_for(n_ * pw), kThreads, 0, s>>>(W, out, pw, beta, X1, p1, coef_, X2 ? X2 : X1,
                                                                     p2, coef_ + size_t(kMaxOrb) * kMaxOrb, L_, n_);
    }
    MCD_LAUNCHED(c_);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // coef_ is reused by the next call
    return e == cudaSuccess ? MCD_OK : cuda_fail(c_, e, "block combine");
  }

  // Orthonormalise the p columns of W (already orthogonal to the earlier
  // blocks) into `out` with deflation: W ~ out * F, returns rank via r.
  int qr(T* W, int p, const std::vector<double>& ref, T* out, int& r, std::vector<double>& F) {
    std::vector<double> G, R, M, F1, G2, R2, M2, F2;
    std::vector<int> piv;
    int st = gram(W, p, W, p, G);
    if (st) return st;
    r = pivoted_cholesky(p, G, ref, sizeof(T) == 8 ? 1e-10 : 1e-5, piv, R);
    if (r == 0) {
      F.clear();
      return MCD_OK;
    }
    factors(p, r, piv, R, M, F1);
    st = combine(W, out, r, 0.0, W, p, M, nullptr, 0, M);
    if (st) return st;
    // second Cholesky QR pass (no deflation): out = out * R2^-1, F = R2 F1
    st = gram(out, r, out, r, G2);
    if (st) return st;
    std::vector<double> one(r, 0.0);
    std::vector<int> piv2;
    const int r2 = pivoted_cholesky(r, G2, std::vector<double>(r, 1.0), 0.0, piv2, R2);
    if (r2 != r) return fail(c_, MCD_E_BREAKDOWN, "band Lanczos: second QR pass lost rank");
    factors(r, r, piv2, R2, M2, F2);
    st = combine(out, W, r, 0.0, out, r, M2, nullptr, 0, M2);   // W temporarily holds the result
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(out, W, size_t(n_) * L_ * sizeof(T), cudaMemcpyDeviceToDevice, c_->stream);
    if (e != cudaSuccess) return cuda_fail(c_, e, "copy block");
    F.assign(size_t(r) * p, 0.0);
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < p; ++j) {
        double s = 0.0;
        for (int k = 0; k < r; ++k) s += F2[size_t(i) * r + k] * F1[size_t(k) * p + j];
        F[size_t(i) * p + j] = s;
      }
    return MCD_OK;
  }

  // Runs the band Lanczos from the start block in buf(0) (L columns).
  int run(int n_blocks, BandRun& out) {
    T* Vprev = B_[1];
    T* Vcur = B_[2];
    T* W = B_[0];
    std::vector<double> G0;
    int st = gram(W, L_, W, L_, G0);
    if (st) return st;
    std::vector<double> ref(L_);
    for (int j = 0; j < L_; ++j) ref[j] = std::sqrt(std::max(G0[size_t(j) * L_ + j], 0.0));
    int p = 0;
    std::vector<double> R0;
    st = qr(W, L_, ref, Vcur, p, R0);
    if (st) return st;
    const int p1 = p;
    std::vector<std::vector<double>> As, Bs;   // A_k (p_k x p_k), B_{k+1} (p_{k+1} x p_k)
    std::vector<int> ps;
    int pprev = 0;
    std::vector<double> Bprev;   // B_k: p_k x p_{k-1}
    int kept = 0;
    for (int k = 0; k < n_blocks && p > 0; ++k) {
      ps.push_back(p);
      if (vall_) {
        if (kept + p > kmax_) return fail(c_, MCD_E_INVALID, "band Lanczos: kept blocks exceed their storage");
        keep_block_kernel<T><<<grid_for(n_ * p), kThreads, 0, c_->stream>>>(Vcur, L_, p, vall_, kmax_, kept, n_);
        MCD_LAUNCHED(c_);
        kept += p;
      }
      st = hv_apply(c_, Vcur, W, p, L_, sizeof(T) == 8 ? MCD_F64 : MCD_F32, nullptr, 0);
      if (st) return st;
      // [W Vcur]^T W in one pass: the norms of W's columns (their size before
      // orthogonalisation, for deflation) and A = Vcur^T W
      std::vector<double> GA;
      st = gram2(W, p, Vcur, p, W, p, GA);
      if (st) return st;
      std::vector<double> refk(p);
      for (int j = 0; j < p; ++j) refk[j] = std::sqrt(std::max(GA[size_t(j) * p + j], 0.0));
      // W -= Vcur A + Vprev B_k^T
      std::vector<double> A(GA.begin() + size_t(p) * p, GA.begin() + size_t(2) * p * p), C1, C2;
      std::vector<double> Bt;   // p_{k-1} x p_k
      if (pprev) {
        Bt.assign(size_t(pprev) * p, 0.0);
        for (int i = 0; i < pprev; ++i)
          for (int j = 0; j < p; ++j) Bt[size_t(i) * p + j] = -Bprev[size_t(j) * pprev + i];
      }
      std::vector<double> mA(A.size());
      for (size_t i = 0; i < A.size(); ++i) mA[i] = -A[i];
      st = combine(W, W, p, 1.0, Vcur, p, mA, pprev ? Vprev : nullptr, pprev, Bt);
      if (st) return st;
      // second Gram-Schmidt pass against the window: [Vcur Vprev]^T W in one pass
      std::vector<double> C12;
      st = gram2(Vcur, p, pprev ? Vprev : nullptr, pprev, W, p, C12);
      if (st) return st;
      C1.assign(C12.begin(), C12.begin() + size_t(p) * p);
      C2.assign(C12.begin() + size_t(p) * p, C12.end());
      std::vector<double> mC1(C1.size()), mC2(C2.size());
      for (size_t i = 0; i < C1.size(); ++i) mC1[i] = -C1[i];
      for (size_t i = 0; i < C2.size(); ++i) mC2[i] = -C2[i];
      st = combine(W, W, p, 1.0, Vcur, p, mC1, pprev ? Vprev : nullptr, pprev, mC2);
      if (st) return st;
      for (size_t i = 0; i < A.size(); ++i) A[i] += C1[i];
      // symmetrise A
      for (int i = 0; i < p; ++i)
        for (int j = i + 1; j < p; ++j) {
          const double v = 0.5 * (A[size_t(i) * p + j] + A[size_t(j) * p + i]);
          A[size_t(i) * p + j] = A[size_t(j) * p + i] = v;
        }
      As.push_back(A);
      if (k + 1 == n_blocks) break;
      int r = 0;
      std::vector<double> Bn;
      st = qr(W, p, refk, Vprev, r, Bn);   // next block written over Vprev
      if (st) return st;
      if (r == 0) break;
      Bs.push_back(Bn);
      Bprev = Bn;
      pprev = p;
      p = r;
      std::swap(Vprev, Vcur);   // Vcur <- new block, Vprev <- old current
    }
    const int nb = int(As.size());
    out.ps.assign(ps.begin(), ps.begin() + nb);
    out.A = As;
    out.B.assign(Bs.begin(), Bs.begin() + std::max(nb - 1, 0));
    out.R0 = R0;
    out.dim = n_;
    if (!vall_) {
      // G from the band matrix itself (band_resolvent): no eigenpairs needed
      int K = 0;
      for (int k = 0; k < nb; ++k) K += ps[k];
      out.K = K;
      return MCD_OK;
    }
    // assemble the block tridiagonal H_eff
    std::vector<int> off(nb + 1, 0);
    for (int k = 0; k < nb; ++k) off[k + 1] = off[k] + ps[k];
    const int K = off[nb];
    std::vector<double> Hm(size_t(K) * K, 0.0);
    for (int k = 0; k < nb; ++k) {
      for (int i = 0; i < ps[k]; ++i)
        for (int j = 0; j < ps[k]; ++j) Hm[size_t(off[k] + i) * K + off[k] + j] = As[k][size_t(i) * ps[k] + j];
      if (k + 1 < nb) {
        const std::vector<double>& Bk = Bs[k];   // p_{k+1} x p_k
        for (int i = 0; i < ps[k + 1]; ++i)
          for (int j = 0; j < ps[k]; ++j) {
            Hm[size_t(off[k + 1] + i) * K + off[k] + j] = Bk[size_t(i) * ps[k] + j];
            Hm[size_t(off[k] + j) * K + off[k + 1] + i] = Bk[size_t(i) * ps[k] + j];
          }
      }
    }
    out.E.assign(K, 0.0);
    const int rows = vall_ ? K : p1;
    std::vector<double> X(size_t(rows) * K, 0.0);
    if (symeig_leading(K, Hm.data(), out.E.data(), rows, X.data()) != 0)
      return fail(c_, MCD_E_NOT_CONVERGED, "band Lanczos: H_eff eigensolver did not converge");
    if (vall_) out.S = X;
    // Q[mu][m] = sum_{i < p1} R0[i][mu] X[i][m]
    out.Q.assign(size_t(L_) * K, 0.0);
    for (int mu = 0; mu < L_; ++mu)
      for (int i = 0; i < p1; ++i) {
        const double rv = R0[size_t(i) * L_ + mu];
        if (rv == 0.0) continue;
        for (int m = 0; m < K; ++m) out.Q[size_t(mu) * K + m] += rv * X[size_t(i) * K + m];
      }
    out.K = K;
    out.dim = n_;
    return MCD_OK;
  }

 private:
  mcd_ctx* c_;
  int L_;
  int64_t n_;
  T* B_[3] = {nullptr, nullptr, nullptr};
  double* part_ = nullptr;
  double* gram_ = nullptr;
  double* coef_ = nullptr;
  int nparts_ = 1;
  double* vall_ = nullptr;
  int kmax_ = 0;
};

// ---- gradient of G with respect to the Hamiltonian's parameters -----------------

// out[r][j] = sum_i A[r][i] M[i][j]  (A: n x k, M: k x cols, fp64, row-major)
__global__ void gemm_rows_kernel(const double* __restrict__ A, int64_t n, int k, const double* __restrict__ M,
                                 int cols, double* out) {
  const int64_t total = n * cols;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols;
    const int j = int(e - r * cols);
    double s = 0.0;
    for (int i = 0; i < k; ++i) s = fma(A[r * k + i], __ldg(M + int64_t(i) * cols + j), s);
    out[e] = s;
  }
}

// r[i] += sum_nu <x| c^(dag)_nu |w_i> F[x][nu]: the start-vector map (start_vec_kernel)
// transposed, one thread per kept ground-state word (deterministic)
__global__ void map_back_kernel(const uint64_t* __restrict__ gw, int64_t ng, const uint64_t* __restrict__ exc,
                                int64_t ne, const double* __restrict__ F, const OrbParams op, double* r) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= ng) return;
  const uint64_t w = gw[i];
  const int n = op.n_sites;
  const uint64_t half = n == 32 ? 0xFFFFFFFFull : ((1ull << n) - 1);
  double acc = 0.0;
  for (int nu = 0; nu < op.L; ++nu) {
    const int sh = op.spin[nu] == 0 ? n + op.site[nu] : op.site[nu];
    const uint64_t bit = 1ull << sh;
    const bool occ = (w & bit) != 0;
    if (occ == bool(op.dagger)) continue;
    const uint64_t x = w ^ bit;
    int64_t lo = 0, len = ne;
    while (len > 1) {
      const int64_t h = len >> 1;
      if (exc[lo + h] <= x) lo += h;
      len -= h;
    }
    if (ne == 0 || exc[lo] != x) continue;
    const uint32_t up = uint32_t(w >> n), dn = uint32_t(w & half);
    const int st = op.site[nu];
    const uint32_t below = (st == 0) ? 0u : (0xFFFFFFFFu >> (32 - st));
    const int before = op.spin[nu] == 0 ? __popc(up & below) : __popc(up) + __popc(dn & below);
    const double f = F[lo * op.L + nu];
    acc += (before & 1) ? -f : f;
  }
  r[i] += acc;
}

// y = a x + b y
__global__ void axpby_kernel(double a, const double* x, double b, double* y, int64_t n) {
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
    y[k] = a * x[k] + b * y[k];
}

// per-block partial sums of a[k] b[k] (summed on the host in block order)
__global__ void __launch_bounds__(kThreads) dot_part_kernel(const double* a, const double* b, int64_t n, double* part) {
  __shared__ double s_red[kThreads / 32];
  double acc = 0.0;
  for (int64_t k = int64_t(blockIdx.x) * kThreads + threadIdx.x; k < n; k += int64_t(gridDim.x) * kThreads)
    acc = fma(a[k], b[k], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
    part[blockIdx.x] = t;
  }
}

// What the gradient takes from one excited space and what it gives back.
struct GradSide {
  const double* z_re;
  const double* z_im;
  int nz;
  const double* g_re;      // [nz][L][L] upstream gradient of Re G
  const double* g_im;      //            and of Im G
  double E0;
  double* d_r;             // device [n kept]: start-vector term, accumulated
  std::vector<double> gt, ge, gu;   // resolvent term, accumulated
  double cE = 0.0;                  // coefficient of dE0, accumulated
};

// The resolvent and start-vector terms of one excited space (sgn = +1
// particle: A = z + E0 - H+; -1 hole: A = z - E0 + H-).  With y_m = V S_m the
// Ritz vectors, beta_mu m(z) = Q_mu m / (z + sgn E0 - sgn E_m) and
// b_mu(z) = sum_m beta_mu m y_m = A^-1 phi_mu on the Krylov space:
//   dG_mu nu = dphi_mu^T b_nu + b_mu^T dphi_nu + sgn b_mu^T dH b_nu - sgn dE0 b_mu^T b_nu.
// Contracted with conj(g): Gamma_mm' = Re sum conj(g_mu nu) beta_mu m beta_nu m'
// gives sgn sum Gamma_mm' y_m^T dH y_m' (one adjoint call, U = V S, V2 = V S
// (sgn Gamma)^T), the dE0 coefficient -sgn tr Gamma, and the vectors
// f_mu = sum_m y_m Re sum (conj(g_mu nu) + conj(g_nu mu)) beta_nu m mapped
// back onto the kept ground-state words by the transposed start-vector map.
int grad_side(mcd_ctx* c, mcd_ctx* sub, const double* vall, int64_t N, const BandRun& run, int L, bool dagger,
              const uint64_t* dgw, int64_t ng, const OrbParams& op, GradSide& gs) {
  const int K = run.K;
  if (K == 0) return MCD_OK;
  const double sgn = dagger ? 1.0 : -1.0;
  const int nz = gs.nz;
  std::vector<double> Gam(size_t(K) * K, 0.0), A(size_t(L) * K, 0.0);
  std::vector<std::complex<double>> beta(size_t(L) * K), Cm(size_t(L) * K);
  for (int iz = 0; iz < nz; ++iz) {
    const std::complex<double> z(gs.z_re[iz], gs.z_im[iz]);
    for (int m = 0; m < K; ++m) {
      const std::complex<double> inv = 1.0 / (z + sgn * gs.E0 - sgn * run.E[m]);
      for (int mu = 0; mu < L; ++mu) beta[size_t(mu) * K + m] = run.Q[size_t(mu) * K + m] * inv;
    }
    const double* gr = gs.g_re + size_t(iz) * L * L;
    const double* gi = gs.g_im + size_t(iz) * L * L;
    // Cm[nu][m] = sum_mu conj(g_mu nu) beta_mu m ; A[mu][m] += Re sum_nu (conj g_mu nu + conj g_nu mu) beta_nu m
    for (int nu = 0; nu < L; ++nu)
      for (int m = 0; m < K; ++m) {
        std::complex<double> acc = 0.0;
        for (int mu = 0; mu < L; ++mu)
          acc += std::complex<double>(gr[mu * L + nu], -gi[mu * L + nu]) * beta[size_t(mu) * K + m];
        Cm[size_t(nu) * K + m] = acc;
      }
    for (int mu = 0; mu < L; ++mu)
      for (int m = 0; m < K; ++m) {
        std::complex<double> acc = 0.0;
        for (int nu = 0; nu < L; ++nu) {
          const std::complex<double> g1(gr[mu * L + nu], -gi[mu * L + nu]), g2(gr[nu * L + mu], -gi[nu * L + mu]);
          acc += (g1 + g2) * beta[size_t(nu) * K + m];
        }
        A[size_t(mu) * K + m] += acc.real();
      }
    for (int m = 0; m < K; ++m)
      for (int mp = 0; mp < K; ++mp) {
        std::complex<double> acc = 0.0;
        for (int nu = 0; nu < L; ++nu) acc += Cm[size_t(nu) * K + m] * beta[size_t(nu) * K + mp];
        Gam[size_t(m) * K + mp] += acc.real();
      }
  }
  for (int m = 0; m < K; ++m) gs.cE += -sgn * Gam[size_t(m) * K + m];
  // M1 = S, M2 = S (sgn Gamma)^T, M3 = S A^T (host, K x K and K x L)
  const std::vector<double>& S = run.S;
  std::vector<double> M2(size_t(K) * K, 0.0), M3(size_t(K) * L, 0.0);
  for (int k = 0; k < K; ++k)
    for (int m = 0; m < K; ++m) {
      const double skm = S[size_t(k) * K + m];
      if (skm == 0.0) continue;
      for (int j = 0; j < K; ++j) M2[size_t(k) * K + j] += skm * sgn * Gam[size_t(j) * K + m];
      for (int mu = 0; mu < L; ++mu) M3[size_t(k) * L + mu] += skm * A[size_t(mu) * K + m];
    }
  cudaStream_t s = c->stream;
  double *dM = nullptr, *U = nullptr, *V2 = nullptr, *F = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dM), sizeof(double) * (size_t(K) * K * 2 + size_t(K) * L), s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&U), sizeof(double) * size_t(N) * K, s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&V2), sizeof(double) * size_t(N) * K, s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&F), sizeof(double) * size_t(N) * L, s);
  auto release = [&]() {
    for (double* q : {dM, U, V2, F})
      if (q) cudaFreeAsync(q, s);
  };
  if (e != cudaSuccess) {
    release();
    return fail(c, MCD_E_OOM, "Green gradient: Ritz-vector buffers");
  }
  e = cudaMemcpyAsync(dM, S.data(), sizeof(double) * K * K, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dM + size_t(K) * K, M2.data(), sizeof(double) * K * K, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dM + 2 * size_t(K) * K, M3.data(), sizeof(double) * K * L, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    gemm_rows_kernel<<<grid_for(N * K), kThreads, 0, s>>>(vall, N, K, dM, K, U);
    gemm_rows_kernel<<<grid_for(N * K), kThreads, 0, s>>>(vall, N, K, dM + size_t(K) * K, K, V2);
    gemm_rows_kernel<<<grid_for(N * L), kThreads, 0, s>>>(vall, N, K, dM + 2 * size_t(K) * K, L, F);
    c->launches += 3;
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "Green gradient: Ritz vectors");
  }
  const int n = c->n;
  std::vector<double> gt(size_t(n) * n), ge(n), gu(n);
  const int64_t before = sub->launches;
  int st = hv_adjoint(sub, U, V2, K, K, MCD_F64, gt.data(), ge.data(), gu.data());
  c->launches += sub->launches - before;
  if (st != MCD_OK) {
    release();
    return fail(c, st, std::string("Green gradient: adjoint: ") + sub->err);
  }
  for (size_t i = 0; i < gt.size(); ++i) gs.gt[i] += gt[i];
  for (int i = 0; i < n; ++i) {
    gs.ge[i] += ge[i];
    gs.gu[i] += gu[i];
  }
  map_back_kernel<<<int((ng + 255) / 256), 256, 0, s>>>(dgw, ng, sub->idx.words, N, F, op, gs.d_r);
  MCD_LAUNCHED(c);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "Green gradient: start-vector term");
}

// ---- target-weight truncation and excited bases on the device -----------------

// Sec. "Further truncation": with w_i = (psi_i / |psi|)^2 sorted descending
// (ties: lower index first), keep the shortest prefix whose weight reaches
// w_t of the total.  Without sorting: tau = the weight at the cut is the
// largest value with sum_{w_i >= tau} w_i >= target, found by bisection over
// the bit patterns of non-negative doubles (ordered like the values); every
// weight above tau is kept and, of those equal to tau, the m of lowest index
// that the target needs.  Every sum is a fixed-order reduction (kTrParts
// block partials summed by one thread), so the cut repeats bit for bit.
constexpr int kTrParts = 1024;
constexpr int kTrThreads = 256;

struct TrState {
  double inv;        // 1 / |psi|
  double total;      // sum of the weights
  double target;     // w_t * total (1 - 1e-15)
  uint64_t lo, hi;   // bisection bounds (bit patterns): S(lo) >= target > S(hi)
  double s_gt;       // sum of the weights above tau
  uint32_t n_eq;     // weights equal to tau
  uint32_t m;        // of those, kept (lowest indices)
};

// mode 0: psi^2; 1: w; 2: w where bits(w) >= (lo + hi) / 2; 3: w > tau (sum)
// and w == tau (count), tau = lo
template <int MODE>
__global__ void __launch_bounds__(kTrThreads) trunc_sum_kernel(const double* __restrict__ psi, int64_t n,
                                                              const TrState* st, double* part, uint32_t* cpart) {
  __shared__ double sd[kTrThreads];
  __shared__ uint32_t sc[kTrThreads];
  const double inv = MODE == 0 ? 1.0 : st->inv;
  uint64_t thr = 0;
  if (MODE == 2) thr = st->lo + (st->hi - st->lo) / 2;
  if (MODE == 3) thr = st->lo;
  double acc = 0.0;
  uint32_t cnt = 0;
  for (int64_t i = int64_t(blockIdx.x) * kTrThreads + threadIdx.x; i < n; i += int64_t(kTrParts) * kTrThreads) {
    const double p = psi[i] * inv;
    const double w = p * p;
    const uint64_t b = uint64_t(__double_as_longlong(w));
    if (MODE <= 1) acc += w;
    if (MODE == 2 && b >= thr) acc += w;
    if (MODE == 3) {
      if (b > thr) acc += w;
      if (b == thr) ++cnt;
    }
  }
  sd[threadIdx.x] = acc;
  sc[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = kTrThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sd[threadIdx.x] += sd[threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sd[0];
    cpart[blockIdx.x] = sc[0];
  }
}

// one thread: the partials in order, then the state update of the mode
template <int MODE>
__global__ void trunc_step_kernel(const double* part, const uint32_t* cpart, TrState* st, double w_t) {
  double s = 0.0;
  uint64_t c = 0;
  for (int b = 0; b < kTrParts; ++b) {
    s += part[b];
    c += cpart[b];
  }
  if (MODE == 0) {
    st->inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  } else if (MODE == 1) {
    st->total = s;
    st->target = w_t * s * (1.0 - 1e-15);
    st->lo = 0;
    st->hi = 0x7FF0000000000000ull;   // +inf: no weight reaches it
  } else if (MODE == 2) {
    const uint64_t mid = st->lo + (st->hi - st->lo) / 2;
    if (st->hi - st->lo > 1) {
      if (s >= st->target) st->lo = mid;
      else st->hi = mid;
    }
  } else {
    const double tau = __longlong_as_double(static_cast<long long>(st->lo));
    st->s_gt = s;
    st->n_eq = uint32_t(c);
    // smallest m with s_gt + m tau >= target (at least one: tau's own state)
    uint64_t m = 1;
    if (tau > 0.0) {
      const double need = (st->target - s) / tau;
      m = need > 1.0 ? uint64_t(ceil(need)) : 1;
      while (m > 1 && s + double(m - 1) * tau >= st->target) --m;
      while (m < c && s + double(m) * tau < st->target) ++m;
    } else {
      m = c;
    }
    st->m = uint32_t(m < c ? m : c);
  }
}

// eq[i] = (w_i == tau)
__global__ void trunc_eq_kernel(const double* __restrict__ psi, int64_t n, const TrState* st, uint32_t* eq) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double p = psi[i] * st->inv;
  eq[i] = uint64_t(__double_as_longlong(p * p)) == st->lo ? 1u : 0u;
}

// keep[i] = w_i > tau, or w_i == tau among the first m such (eqpos = exclusive scan of eq)
__global__ void trunc_keep_kernel(const double* __restrict__ psi, int64_t n, const TrState* st,
                                  const uint32_t* eqpos, uint32_t* keep) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double p = psi[i] * st->inv;
  const uint64_t b = uint64_t(__double_as_longlong(p * p));
  keep[i] = (b > st->lo || (b == st->lo && eqpos[i] < st->m)) ? 1u : 0u;
}

// the kept states in index order: basis index, word, psi value
__global__ void trunc_compact_kernel(const double* __restrict__ psi, const uint64_t* __restrict__ words, int64_t n,
                                     const uint32_t* keep, const uint32_t* pos, uint32_t* idx, uint64_t* kw,
                                     double* kc) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n || !keep[i]) return;
  const uint32_t p = pos[i];
  idx[p] = uint32_t(i);
  kw[p] = words[i];
  kc[p] = psi[i];
}

__global__ void __launch_bounds__(kTrThreads) sq_part_kernel(const double* __restrict__ v, int64_t n, double* part) {
  __shared__ double sd[kTrThreads];
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * kTrThreads + threadIdx.x; i < n; i += int64_t(kTrParts) * kTrThreads)
    acc += v[i] * v[i];
  sd[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kTrThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sd[threadIdx.x] += sd[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sd[0];
}

__global__ void scale_vec_kernel(double* v, int64_t n, const double* part) {
  __shared__ double f;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < kTrParts; ++b) s += part[b];
    f = 1.0 / sqrt(s);
  }
  __syncthreads();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    v[i] *= f;
}

// Kept ground state on the device: idx (ascending basis indices), words and
// renormalised coefficients of the kept states; kn = |P psi|^2 / |psi|^2.
struct KeptDev {
  uint32_t* idx = nullptr;
  uint64_t* words = nullptr;
  double* coef = nullptr;
  int64_t n = 0;
  double kn = 0.0;
  cudaStream_t s = nullptr;
  ~KeptDev() {
    for (void* p : {static_cast<void*>(idx), static_cast<void*>(words), static_cast<void*>(coef)})
      if (p) cudaFreeAsync(p, s);
  }
};

int kept_ground_state_dev(mcd_ctx* c, double w_t, KeptDev& out) {
  const int64_t N = c->idx.n;
  cudaStream_t s = c->stream;
  out.s = s;
  const double* psi = c->gs_psi;
  // work: TrState | partials | counts | eq/eqpos | keep | pos
  const size_t off_part = 64, off_cnt = off_part + sizeof(double) * kTrParts,
               off_eq = off_cnt + sizeof(uint32_t) * kTrParts + 64;
  const size_t off_keep = off_eq + sizeof(uint32_t) * size_t(N) + 64, off_pos = off_keep + sizeof(uint32_t) * size_t(N) + 64;
  unsigned char* wk = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&wk), off_pos + sizeof(uint32_t) * size_t(N) + 64, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "truncation work");
  struct Free {
    void* p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } guard{wk, s};
  TrState* st = reinterpret_cast<TrState*>(wk);
  double* part = reinterpret_cast<double*>(wk + off_part);
  uint32_t* cpart = reinterpret_cast<uint32_t*>(wk + off_cnt);
  uint32_t* eq = reinterpret_cast<uint32_t*>(wk + off_eq);
  uint32_t* keep = reinterpret_cast<uint32_t*>(wk + off_keep);
  uint32_t* pos = reinterpret_cast<uint32_t*>(wk + off_pos);
  trunc_sum_kernel<0><<<kTrParts, kTrThreads, 0, s>>>(psi, N, st, part, cpart);
  trunc_step_kernel<0><<<1, 1, 0, s>>>(part, cpart, st, w_t);
  trunc_sum_kernel<1><<<kTrParts, kTrThreads, 0, s>>>(psi, N, st, part, cpart);
  trunc_step_kernel<1><<<1, 1, 0, s>>>(part, cpart, st, w_t);
  c->launches += 4;
  for (int it = 0; it < 64; ++it) {
    trunc_sum_kernel<2><<<kTrParts, kTrThreads, 0, s>>>(psi, N, st, part, cpart);
    trunc_step_kernel<2><<<1, 1, 0, s>>>(part, cpart, st, w_t);
    c->launches += 2;
  }
  trunc_sum_kernel<3><<<kTrParts, kTrThreads, 0, s>>>(psi, N, st, part, cpart);
  trunc_step_kernel<3><<<1, 1, 0, s>>>(part, cpart, st, w_t);
  const int g = int((N + 255) / 256);
  trunc_eq_kernel<<<g, 256, 0, s>>>(psi, N, st, eq);
  c->launches += 3;
  e = scan_u32(c, eq, eq, N, s);
  if (e == cudaSuccess) {
    trunc_keep_kernel<<<g, 256, 0, s>>>(psi, N, st, eq, keep);
    MCD_LAUNCHED(c);
    e = scan_u32(c, keep, pos, N, s);
  }
  uint32_t last_pos = 0, last_keep = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&last_pos, pos + N - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&last_keep, keep + N - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "truncation");
  const int64_t nk = int64_t(last_pos) + last_keep;
  if (nk < 1) return fail(c, MCD_E_BREAKDOWN, "truncation kept no state (zero ground state)");
  e = cudaMallocAsync(reinterpret_cast<void**>(&out.idx), sizeof(uint32_t) * size_t(nk), s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&out.words), sizeof(uint64_t) * size_t(nk), s);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&out.coef), sizeof(double) * size_t(nk), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "kept ground state");
  out.n = nk;
  trunc_compact_kernel<<<g, 256, 0, s>>>(psi, c->idx.words, N, keep, pos, out.idx, out.words, out.coef);
  // |P psi|^2 (psi as stored), then the kept coefficients renormalised
  sq_part_kernel<<<kTrParts, kTrThreads, 0, s>>>(out.coef, nk, part);
  c->launches += 2;
  double kn_raw = 0.0, inv = 0.0;
  std::vector<double> hp(kTrParts);
  e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * kTrParts, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&inv, &st->inv, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) {
    scale_vec_kernel<<<int(std::min<int64_t>((nk + 255) / 256, 4096)), 256, 0, s>>>(out.coef, nk, part);
    MCD_LAUNCHED(c);
    e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "kept ground state");
  for (double v : hp) kn_raw += v;
  out.kn = kn_raw * inv * inv;
  return MCD_OK;
}

// The excited basis (Sec. "Subspace of the Green function") on the device:
// the distinct words c^dag_mu w (dagger) or c_mu w over the kept words w and
// the orbitals (all of one spin) in orbmask, ascending.
__global__ void exc_count_kernel(const uint64_t* __restrict__ gw, int64_t ng, uint64_t orbmask, int dagger,
                                 uint32_t* cnt) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= ng) return;
  const uint64_t w = gw[i];
  cnt[i] = uint32_t(__popcll(dagger ? (~w & orbmask) : (w & orbmask)));
}

__global__ void exc_write_kernel(const uint64_t* __restrict__ gw, int64_t ng, uint64_t orbmask, int dagger,
                                 const uint32_t* pos, uint64_t* out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= ng) return;
  const uint64_t w = gw[i];
  uint64_t m = dagger ? (~w & orbmask) : (w & orbmask);
  uint32_t p = pos[i];
  while (m) {
    const uint64_t b = m & (~m + 1);
    out[p++] = w ^ b;
    m ^= b;
  }
}

int excited_basis_dev(mcd_ctx* c, const uint64_t* gw, int64_t ng, uint64_t orbmask, bool dagger, uint64_t** exc,
                      int64_t* nexc) {
  *exc = nullptr;
  *nexc = 0;
  cudaStream_t s = c->stream;
  uint32_t* cnt = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&cnt), sizeof(uint32_t) * size_t(ng) + 16, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "excited basis counts");
  const int g = int((ng + 255) / 256);
  exc_count_kernel<<<g, 256, 0, s>>>(gw, ng, orbmask, dagger ? 1 : 0, cnt);
  MCD_LAUNCHED(c);
  uint32_t last_cnt = 0, last_pos = 0;
  e = cudaMemcpyAsync(&last_cnt, cnt + ng - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = scan_u32(c, cnt, cnt, ng, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&last_pos, cnt + ng - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const int64_t total = int64_t(last_pos) + last_cnt;
  uint64_t* cand = nullptr;
  if (e == cudaSuccess && total > 0) e = cudaMallocAsync(reinterpret_cast<void**>(&cand), sizeof(uint64_t) * size_t(total), s);
  if (e == cudaSuccess && total > 0) {
    exc_write_kernel<<<g, 256, 0, s>>>(gw, ng, orbmask, dagger ? 1 : 0, cnt, cand);
    MCD_LAUNCHED(c);
    e = cudaGetLastError();
  }
  cudaFreeAsync(cnt, s);
  if (e != cudaSuccess) {
    if (cand) cudaFreeAsync(cand, s);
    return cuda_fail(c, e, "excited basis candidates");
  }
  if (total == 0) return MCD_OK;
  const int st = sort_unique_device(c, cand, total, 2 * c->n, exc, nexc);
  cudaFreeAsync(cand, s);
  return st;
}

template <typename T>
int one_side(mcd_ctx* c, const uint64_t* dgw, const double* dgc, int64_t ng, const int* site, const int* spin,
             int L, bool dagger, int n_blocks, BandRun& out, GradSide* gs = nullptr) {
  const int n = c->n;
  const int sp = spin[0];
  cudaStream_t s = c->stream;
  // excited basis: c^dag_mu w or c_mu w over the kept w, on the device
  uint64_t orbmask = 0;
  for (int mu = 0; mu < L; ++mu) orbmask |= 1ull << (spin[mu] == 0 ? n + site[mu] : site[mu]);
  uint64_t* exc = nullptr;
  int64_t nexc = 0;
  int st = excited_basis_dev(c, dgw, ng, orbmask, dagger, &exc, &nexc);
  if (st != MCD_OK) return st;
  struct FreeExc {
    uint64_t*& p;
    cudaStream_t s;
    ~FreeExc() {
      if (p) cudaFreeAsync(p, s);
    }
  } free_exc{exc, s};
  out.dim = nexc;
  if (nexc == 0) {
    out.K = 0;
    return MCD_OK;
  }
  const int dnu = dagger ? 1 : -1;
  const int nup = c->n_up + (sp == 0 ? dnu : 0), ndn = c->n_dn + (sp == 1 ? dnu : 0);
  mcd_ctx* sub = nullptr;
  st = mcd_create(&sub, c->device, c->stream);
  if (st) return fail(c, st, "band Lanczos: internal context");
  struct Guard {
    mcd_ctx* p;
    ~Guard() { mcd_destroy(p); }
  } guard{sub};
  sub->hv_algo = c->hv_algo;
  sub->hv_cache = c->hv_cache;
  sub->timing = c->timing;   // its products count in this context's kernel times
  sub->tm = c->tm;
  sub->tm_borrowed = true;
  st = mcd_set_hamiltonian(sub, n, c->t.data(), c->eps.data(), c->U.data(), n, nup, ndn);
  if (st == MCD_OK) st = mcd_set_basis_device(sub, exc, nexc);
  if (st != MCD_OK) return fail(c, st, std::string("band Lanczos: excited space: ") + sub->err);
  cudaFreeAsync(exc, s);
  exc = nullptr;
  c->launches += sub->launches;
  const int64_t before = sub->launches;
  cudaError_t e = cudaSuccess;
  BandLanczos<T> bl(sub, L);
  st = bl.alloc();
  double* vall = nullptr;
  const int kmax = n_blocks * L;
  if (st == MCD_OK && gs) {
    if (cudaMallocAsync(reinterpret_cast<void**>(&vall), sizeof(double) * size_t(nexc) * kmax, s) != cudaSuccess) {
      vall = nullptr;
      st = fail(c, MCD_E_OOM, "Green gradient: the Krylov blocks of an excited space do not fit");
    } else {
      bl.keep_blocks(vall, kmax);
    }
  }
  OrbParams op;
  std::memset(&op, 0, sizeof(op));
  if (st == MCD_OK) {
    op.L = L;
    op.dagger = dagger ? 1 : 0;
    op.n_sites = n;
    for (int mu = 0; mu < L; ++mu) {
      op.site[mu] = site[mu];
      op.spin[mu] = spin[mu];
    }
    const int64_t ne = nexc;
    start_vec_kernel<T><<<int((ne + 255) / 256), 256, 0, s>>>(sub->idx.words, ne, dgw, dgc, ng, bl.buf(0), L, op);
    MCD_LAUNCHED(sub);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(c, e, "start vectors");
  }
  if (st == MCD_OK) {
    st = bl.run(n_blocks, out);
    if (st == MCD_OK) st = take_wait_errors(sub);   // a product whose bounded wait gave up is incomplete
    if (st != MCD_OK) c->err = sub->err;
  }
  c->launches += sub->launches - before;
  if (st == MCD_OK && gs) {
    const int64_t b2 = sub->launches;
    st = grad_side(c, sub, vall, nexc, out, L, dagger, dgw, ng, op, *gs);
    c->launches += sub->launches - b2;
  }
  if (vall) cudaFreeAsync(vall, s);
  return st;
}

// argument checks shared by the Green function and its gradient
int check_orbitals(mcd_ctx* c, const int* site, const int* spin, int L, int n_blocks, double w_t) {
  if (!c->gs_valid) return fail(c, MCD_E_STATE, "no ground state: call mcd_lanczos_ground first");
  if (L < 1 || L > kMaxOrb) return fail(c, MCD_E_INVALID, "need 1 <= L <= 64 orbitals");
  for (int mu = 0; mu < L; ++mu) {
    if (site[mu] < 0 || site[mu] >= c->n || (spin[mu] != 0 && spin[mu] != 1))
      return fail(c, MCD_E_INVALID, "orbital (site, spin) out of range");
    if (spin[mu] != spin[0])
      return fail(c, MCD_E_INVALID, "orbitals must share one spin (G is block diagonal in spin)");
  }
  if (n_blocks < 1) return fail(c, MCD_E_INVALID, "n_block_iter must be >= 1");
  if (!(w_t > 0.0 && w_t <= 1.0)) return fail(c, MCD_E_INVALID, "w_t must be in (0, 1]");
  return MCD_OK;
}

// The device truncation's result on the host (the Green gradient works on
// the kept words there): psi = the normalised ground state, keep = the kept
// basis indices (ascending), kw / kc = their words and renormalised
// coefficients.
int kept_to_host(mcd_ctx* c, const KeptDev& kd, std::vector<double>& psi, std::vector<int64_t>& keep,
                 std::vector<uint64_t>& kw, std::vector<double>& kc) {
  const int64_t N = c->idx.n, nk = kd.n;
  cudaStream_t s = c->stream;
  psi.resize(N);
  std::vector<uint32_t> idx(nk);
  kw.resize(nk);
  kc.resize(nk);
  cudaError_t e = cudaMemcpyAsync(psi.data(), c->gs_psi, sizeof(double) * N, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(idx.data(), kd.idx, sizeof(uint32_t) * nk, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(kw.data(), kd.words, sizeof(uint64_t) * nk, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(kc.data(), kd.coef, sizeof(double) * nk, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "kept ground state to host");
  keep.assign(idx.begin(), idx.end());
  double nn = 0.0;
  for (double v : psi) nn += v * v;
  const double inv = 1.0 / std::sqrt(nn);
  for (double& v : psi) v *= inv;
  return MCD_OK;
}

}  // namespace

int band_lanczos_green(mcd_ctx* c, const int* site, const int* spin, int L, int n_blocks, double w_t, int dtype,
                       const double* z_re, const double* z_im, int nz, double* G_re, double* G_im,
                       int64_t* dim_plus, int64_t* dim_minus) {
  int st0 = check_orbitals(c, site, spin, L, n_blocks, w_t);
  if (st0 != MCD_OK) return st0;
  KeptDev kd;
  st0 = kept_ground_state_dev(c, w_t, kd);
  if (st0 != MCD_OK) return st0;
  BandRun plus, minus;
  int st = dtype == MCD_F64 ? one_side<double>(c, kd.words, kd.coef, kd.n, site, spin, L, true, n_blocks, plus)
                            : one_side<float>(c, kd.words, kd.coef, kd.n, site, spin, L, true, n_blocks, plus);
  if (st == MCD_OK)
    st = dtype == MCD_F64 ? one_side<double>(c, kd.words, kd.coef, kd.n, site, spin, L, false, n_blocks, minus)
                          : one_side<float>(c, kd.words, kd.coef, kd.n, site, spin, L, false, n_blocks, minus);
  if (st != MCD_OK) return st;
  if (dim_plus) *dim_plus = plus.dim;
  if (dim_minus) *dim_minus = minus.dim;
  // G+ = R0+^T (z + E0 - H+_eff)^{-1} R0+ and G- = R0-^T (z - E0 + H-_eff)^{-1} R0-,
  // the Lehmann sums of App. C over the eigenpairs of each H_eff
  const double E0 = c->gs_E0;
  std::fill(G_re, G_re + size_t(nz) * L * L, 0.0);
  std::fill(G_im, G_im + size_t(nz) * L * L, 0.0);
  if (!band_resolvent(plus, L, E0, true, z_re, z_im, nz, G_re, G_im) ||
      !band_resolvent(minus, L, E0, false, z_re, z_im, nz, G_re, G_im))
    return fail(c, MCD_E_BREAKDOWN, "band Lanczos: singular block of z - H_eff");
  return MCD_OK;
}

// Gradient of S = sum_{z,mu,nu} gR Re G_mu nu(z) + gI Im G_mu nu(z) with respect
// to (t_ij per bond, eps_i, U_i), G as mcd_band_lanczos_green computes it (the
// Krylov resolvent in the truncated excited spaces), the kept ground-state
// words held fixed.  Besides the two excited-space terms (grad_side):
//   dE0 = <Omega|dH|Omega> (Hellmann-Feynman) with the accumulated coefficient;
//   the start vectors phi = c^(dag) P Omega / |P Omega| depend on Omega: the
//   map-back r (on the kept words) becomes, through the renormalisation,
//   rt = P (r - Omega_t <Omega_t|r>) / |P Omega|, and with the first-order
//   response dOmega = -(H - E0)^+ (dH - dE0) Omega the term is -lambda^T dH Omega,
//   lambda = (H - E0)^+ rt_perp, found by conjugate gradients on the
//   complement of Omega.  One last adjoint call takes u = cE Omega - lambda.
int green_gradient(mcd_ctx* c, const int* site, const int* spin, int L, int n_blocks, double w_t,
                   const double* z_re, const double* z_im, int nz, const double* g_re, const double* g_im,
                   double* grad_t, double* grad_eps, double* grad_U, double cg_tol, int* cg_iters) {
  int st = check_orbitals(c, site, spin, L, n_blocks, w_t);
  if (st != MCD_OK) return st;
  std::vector<double> psi, kc;
  std::vector<int64_t> keep;
  std::vector<uint64_t> kw;
  KeptDev kd;
  st = kept_ground_state_dev(c, w_t, kd);
  if (st == MCD_OK) st = kept_to_host(c, kd, psi, keep, kw, kc);
  if (st != MCD_OK) return st;
  const double kn = kd.kn;
  const int n = c->n;
  const int64_t N = c->idx.n, nk = int64_t(keep.size());
  cudaStream_t s = c->stream;
  GradSide gs;
  gs.z_re = z_re;
  gs.z_im = z_im;
  gs.nz = nz;
  gs.g_re = g_re;
  gs.g_im = g_im;
  gs.E0 = c->gs_E0;
  gs.gt.assign(size_t(n) * n, 0.0);
  gs.ge.assign(n, 0.0);
  gs.gu.assign(n, 0.0);
  double* buf = nullptr;   // d_r [nk] | b, lam, r, p, q, u [N each] | partials [kParts]
  const int kParts = device_sms() * 4;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), sizeof(double) * (size_t(nk) + 6 * size_t(N) + kParts), s);
  if (e != cudaSuccess) return fail(c, MCD_E_OOM, "Green gradient: work vectors");
  struct Free {
    double* p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } guard{buf, s};
  gs.d_r = buf;
  double* vb = buf + nk;
  double* lam = vb + N;
  double* r = lam + N;
  double* pv = r + N;
  double* q = pv + N;
  double* u = q + N;
  double* part = u + N;
  e = cudaMemsetAsync(buf, 0, sizeof(double) * (size_t(nk) + 6 * size_t(N)), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Green gradient: clear");
  BandRun plus, minus;
  st = one_side<double>(c, kd.words, kd.coef, kd.n, site, spin, L, true, n_blocks, plus, &gs);
  if (st == MCD_OK) st = one_side<double>(c, kd.words, kd.coef, kd.n, site, spin, L, false, n_blocks, minus, &gs);
  if (st != MCD_OK) return st;
  // start-vector term through the renormalised truncation, on the full basis
  std::vector<double> rk(nk), b(N, 0.0);
  e = cudaMemcpyAsync(rk.data(), gs.d_r, sizeof(double) * nk, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Green gradient: start-vector term");
  double kr = 0.0;
  for (int64_t i = 0; i < nk; ++i) kr += kc[i] * rk[i];
  const double pn = std::sqrt(kn);
  for (int64_t i = 0; i < nk; ++i) b[keep[i]] = (rk[i] - kc[i] * kr) / pn;
  double ob = 0.0;
  for (int64_t i = 0; i < N; ++i) ob += psi[i] * b[i];
  for (int64_t i = 0; i < N; ++i) b[i] -= ob * psi[i];
  e = cudaMemcpyAsync(vb, b.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Green gradient: right-hand side");
  const double* om = c->gs_psi;
  const int vg = grid_for(N);
  auto dot = [&](const double* x, const double* y, double& out) -> int {
    dot_part_kernel<<<kParts, kThreads, 0, s>>>(x, y, N, part);
    MCD_LAUNCHED(c);
    std::vector<double> h(kParts);
    cudaError_t er = cudaMemcpyAsync(h.data(), part, sizeof(double) * kParts, cudaMemcpyDeviceToHost, s);
    if (er == cudaSuccess) er = cudaStreamSynchronize(s);
    if (er != cudaSuccess) return cuda_fail(c, er, "Green gradient: dot");
    out = 0.0;
    for (double v : h) out += v;
    return MCD_OK;
  };
  auto axpby = [&](double a, const double* x, double bb, double* y) {
    axpby_kernel<<<vg, kThreads, 0, s>>>(a, x, bb, y, N);
    MCD_LAUNCHED(c);
  };
  // conjugate gradients for (H - E0) lam = b on the complement of Omega
  const double E0 = c->gs_E0;
  double rr = 0.0;
  e = cudaMemcpyAsync(r, vb, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pv, vb, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Green gradient: CG start");
  if ((st = dot(r, r, rr)) != MCD_OK) return st;
  const double bnorm = std::sqrt(rr);
  int it = 0;
  bool conv = bnorm == 0.0;
  const int max_it = 20000;
  for (; !conv && it < max_it; ++it) {
    st = hv_apply(c, pv, q, 1, 1, MCD_F64, nullptr, 0);
    if (st != MCD_OK) return st;
    axpby(-E0, pv, 1.0, q);
    double oq = 0.0, pq = 0.0, rn = 0.0, orr = 0.0;
    if ((st = dot(om, q, oq)) != MCD_OK) return st;
    axpby(-oq, om, 1.0, q);
    if ((st = dot(pv, q, pq)) != MCD_OK) return st;
    if (!(pq > 0.0)) return fail(c, MCD_E_BREAKDOWN, "Green gradient: H - E0 not positive on the complement");
    const double alpha = rr / pq;
    axpby(alpha, pv, 1.0, lam);
    axpby(-alpha, q, 1.0, r);
    if ((st = dot(om, r, orr)) != MCD_OK) return st;
    axpby(-orr, om, 1.0, r);
    if ((st = dot(r, r, rn)) != MCD_OK) return st;
    if (std::sqrt(rn) <= cg_tol * bnorm) conv = true;
    axpby(1.0, r, rn / rr, pv);
    rr = rn;
  }
  if (cg_iters) *cg_iters = it;
  // last adjoint: u = cE Omega - lam against Omega
  axpby(gs.cE, om, 0.0, u);
  axpby(-1.0, lam, 1.0, u);
  std::vector<double> gt(size_t(n) * n), ge(n), gu(n);
  st = hv_adjoint(c, u, om, 1, 1, MCD_F64, gt.data(), ge.data(), gu.data());
  if (st != MCD_OK) return st;
  for (int i = 0; i < n * n; ++i) grad_t[i] = gs.gt[i] + gt[i];
  for (int i = 0; i < n; ++i) {
    grad_eps[i] = gs.ge[i] + ge[i];
    grad_U[i] = gs.gu[i] + gu[i];
  }
  if (!conv) return fail(c, MCD_E_NOT_CONVERGED, "Green gradient: conjugate gradients did not converge");
  return MCD_OK;
}

}  // namespace mcd
