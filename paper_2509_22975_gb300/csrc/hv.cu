// y = H~ x without storing H~ (App. B: out-of-basis targets are discarded,
// which is the projected matrix of the truncated basis).
//
// H = H_up + H_dn + D with D diagonal (Eq. (1)).  A down-spin hop keeps the
// up word, an up-spin hop keeps the down word, so
//   pass B (dn-major blocks, states sharing a dn word): y[perm k] = sum over
//     up-spin hops of t_ij sign x[target]          (stores every row once)
//   pass A (up-major blocks = basis order):           y[k] += D_k x[k] +
//     sum over dn-spin hops of t_ij sign x[target]
// Within a pass every hop target lies in the state's own block, whose minor
// words a CTA stages in shared memory and binary-searches.  H~ is real
// symmetric, so row k is gathered from the targets of the hops of state k
// (pull form: no atomics, each row written by one thread group).
//
// Thread mapping: a group of G lanes per state; lane g owns columns
// [g*VEC, g*VEC+VEC) of each row and evaluates bonds g, g+G, ...; found
// targets are broadcast within the group by shuffles, then every lane
// gathers its column chunk of the target row (coalesced 16-byte loads when
// the rows are aligned).
#include <atomic>
#include <algorithm>
#include <cmath>

#include "hv_common.cuh"

namespace mcd {
namespace {

constexpr int kThreads = 256;
constexpr int kBitmapMaxSites = 16;            // 2^16-bit bitmap = 8 KiB of shared memory
constexpr int kStageXBytes = 52 * 1024;        // x staging area of the bitmap kernel
constexpr int kStageX1Bytes = 20 * 1024;       // x staging area of the single-column kernel
constexpr int kStageXcBytes = 52 * 1024;       // shared memory of the multi-column kernel
constexpr int kLcCap = 48;                     // found hops per state in its list

// ---------------------------------------------------------------------------------
template <typename T, int VEC, int G, bool PASS_A, bool DOT>
__global__ void __launch_bounds__(kThreads) hv_block_kernel(const HvArgs a, const HamParams hp) {
  extern __shared__ uint32_t s_minor[];
  __shared__ uint32_t s_off[kItem + 2];
  __shared__ uint32_t s_major[kItem + 1];
  __shared__ uint32_t s_mask[kMaxBonds], s_betw[kMaxBonds];
  __shared__ float s_thi[kMaxBonds], s_tlo[kMaxBonds];
  __shared__ double s_t64[kMaxBonds];
  __shared__ int s_nb, s_st0, s_staged;
  __shared__ double s_red[kThreads / 32];

  const Layout& L = a.L;
  const int item = blockIdx.x;
  const int64_t k0 = int64_t(item) * kItem;
  const int64_t k1 = (k0 + kItem < L.n ? k0 + kItem : L.n);
  const int nbonds = hp.n_bonds;
  for (int b = threadIdx.x; b < nbonds; b += kThreads) {
    s_mask[b] = hp.bonds[b].mask;
    s_betw[b] = hp.bonds[b].between;
    s_thi[b] = hp.bonds[b].t_hi;
    s_tlo[b] = hp.bonds[b].t_lo;
    s_t64[b] = hp.bonds[b].t;
  }
  if (threadIdx.x == 0) {
    const uint32_t b0 = L.item_blk[item];
    uint32_t b1 = L.item_blk[item + 1];
    if (b1 == uint32_t(L.nblk) || L.blk_off[b1] == uint32_t(k1)) b1 -= 1;
    s_nb = int(b1 - b0 + 1);
    s_st0 = int(L.blk_off[b0]);
    const int st1 = int(L.blk_off[b1 + 1]);
    s_staged = (st1 - s_st0) <= kStageWords;
  }
  __syncthreads();
  const int nb = s_nb, st0 = s_st0;
  const uint32_t b0 = L.item_blk[item];
  for (int j = threadIdx.x; j <= nb; j += kThreads) {
    s_off[j] = L.blk_off[b0 + j];
    if (j < nb) s_major[j] = L.blk_major[b0 + j];
  }
  __syncthreads();
  const int st1 = int(s_off[nb]);
  const uint32_t* mw;
  int mbase;   // mw[pos - mbase] = minor word of layout position pos
  if (s_staged) {
    for (int p = threadIdx.x; p < st1 - st0; p += kThreads) s_minor[p] = L.minor[st0 + p];
    mw = s_minor;
    mbase = st0;
    __syncthreads();
  } else {
    mw = L.minor + st0;
    mbase = st0;
  }

  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const int lane = threadIdx.x & 31;
  const int g = lane % G;
  const int group = threadIdx.x / G;
  constexpr int kGroups = kThreads / G;
  const unsigned gmask = 0xffffffffu;   // every lane runs the same trip counts
  const int ncols = a.ncols, ld = a.ld;
  const int ctile = G * VEC;
  using C = ChunkOf<T, VEC>;
  double dot_acc = 0.0;

  // every group runs the same number of rounds so that shuffles stay uniform
  const int rounds = (kItem + kGroups - 1) / kGroups;
  for (int r = 0; r < rounds; ++r) {
    const int64_t k = k0 + int64_t(r) * kGroups + group;
    const bool live = k < k1;
    // block of state k among the staged blocks
    int j = 0;
    if (live) {
      int lo = 0, len = nb;
      while (len > 1) {
        const int half = len >> 1;
        if (s_off[lo + half] <= uint32_t(k)) lo += half;
        len -= half;
      }
      j = lo;
    }
    const int bbase = live ? int(s_off[j]) : 0;
    const int bend = live ? int(s_off[j + 1]) : 0;
    const uint32_t major = live ? s_major[j] : 0u;
    const uint32_t m = live ? mw[k - mbase] : 0u;
    const int64_t out_row = live ? (PASS_A ? k : int64_t(L.perm[k])) : 0;

    for (int c0 = 0; c0 < ncols; c0 += ctile) {
      const int col = c0 + g * VEC;
      const int cvalid = ncols - col;
      Acc<T> acc[VEC];
#pragma unroll
      for (int c = 0; c < VEC; ++c) acc[c].zero();
      for (int bb = 0; bb < nbonds; bb += G) {
        const int b = bb + g;
        int row = -1;
        Coef<T> cf{T(0), T(0)};
        if (live && b < nbonds) {
          const uint32_t mk = s_mask[b];
          if (__popc(m & mk) == 1) {
            const uint32_t m2 = m ^ mk;
            const int q = find_sorted(mw, bbase - mbase, bend - mbase, m2);
            if (q >= 0) {
              const int pos = q + mbase;
              row = PASS_A ? pos : int(L.perm[pos]);
              cf = bond_coef<T>(s_thi, s_tlo, s_t64, b, __popc(m & s_betw[b]) & 1);
            }
          }
        }
        if (G == 1) {
          if (row >= 0 && cvalid > 0) {
            T xv[VEC];
            C::load(x + int64_t(row) * ld + col, cvalid, xv);
#pragma unroll
            for (int c = 0; c < VEC; ++c) acc[c].fma(cf.hi, cf.lo, xv[c]);
          }
        } else {
#pragma unroll
          for (int s = 0; s < G; ++s) {
            const int rr = __shfl_sync(gmask, row, s, G);
            const T ch = __shfl_sync(gmask, cf.hi, s, G);
            const T cl = __shfl_sync(gmask, cf.lo, s, G);
            if (rr >= 0 && cvalid > 0) {
              T xv[VEC];
              C::load(x + int64_t(rr) * ld + col, cvalid, xv);
#pragma unroll
              for (int c = 0; c < VEC; ++c) acc[c].fma(ch, cl, xv[c]);
            }
          }
        }
      }
      if (live && cvalid > 0) {
        T out[VEC];
        if (PASS_A) {
          const Coef<T> dc = diag_coef<T>(hp, major, m);
          T xv[VEC], yv[VEC];
          C::load(x + k * ld + col, cvalid, xv);
          C::load(y + k * ld + col, cvalid, yv);
#pragma unroll
          for (int c = 0; c < VEC; ++c) {
            acc[c].fma(dc.hi, dc.lo, xv[c]);
            out[c] = acc[c].value() + yv[c];
          }
          if (DOT) dot_acc += double(xv[0]) * double(out[0]);
        } else {
#pragma unroll
          for (int c = 0; c < VEC; ++c) out[c] = acc[c].value();
        }
        C::store(y + out_row * ld + col, cvalid, out);
      }
    }
  }

  if (DOT) {
    // per-CTA partial of sum_k x[k] y[k]; the last CTA to finish sums the
    // partials in a fixed order (deterministic) into *dot_out.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot_acc += __shfl_xor_sync(0xffffffffu, dot_acc, o);
    if (lane == 0) s_red[threadIdx.x >> 5] = dot_acc;
    __syncthreads();
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) s += s_red[w];
      a.dot_partials[blockIdx.x] = s;
      __threadfence();
      const unsigned t = atomicAdd(a.ticket, 1u);
      s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
      double s = 0.0;
      for (int i = threadIdx.x; i < int(gridDim.x); i += kThreads) s += __ldcg(a.dot_partials + i);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) s_red[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) tot += s_red[w];
        *a.dot_out = tot;
        *a.ticket = 0u;
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Bitmap variant for n_sites <= 16.  For each block (states sharing the major
// word) the CTA marks the minor words of all its states in a 2^n-bit shared
// bitmap and stores, per 32-bit bitmap word, the block-local index of the
// first state in it.  A hop target m2 is then in the basis iff its bit is set,
// and its block-local index is pre[m2 >> 5] + popc(bits of that word below
// m2): one shared load decides membership, a second gives the position.  The
// x rows of the block are staged in shared memory when they fit, so the
// gathers of found targets are shared loads too.  The CTA clears the bits it
// set before moving to the next block.
template <typename T, int VEC, int G, bool PASS_A, bool DOT>
__global__ void __launch_bounds__(kThreads) hv_bitmap_kernel(const HvArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ uint32_t s_b0, s_b1;
  __shared__ double s_red[kThreads / 32];
  const int nbp = a.nbp;
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(s_dyn);
  uint32_t* s_betw = s_mask + nbp;
  float* s_thi = reinterpret_cast<float*>(s_betw + nbp);
  float* s_tlo = s_thi + nbp;
  double* s_t64 = reinterpret_cast<double*>(s_tlo + nbp);
  uint32_t* bm = reinterpret_cast<uint32_t*>(s_dyn + a.off_bm);
  uint16_t* pre = reinterpret_cast<uint16_t*>(s_dyn + a.off_pre);
  T* xs = reinterpret_cast<T*>(s_dyn + a.off_xs);

  const Layout& L = a.L;
  const int item = blockIdx.x;
  const int64_t k0 = int64_t(item) * kItem;
  const int64_t k1 = (k0 + kItem < L.n) ? k0 + kItem : L.n;
  const int nbonds = hp.n_bonds;
  for (int b = threadIdx.x; b < nbonds; b += kThreads) {
    s_mask[b] = hp.bonds[b].mask;
    s_betw[b] = hp.bonds[b].between;
    s_thi[b] = hp.bonds[b].t_hi;
    s_tlo[b] = hp.bonds[b].t_lo;
    s_t64[b] = hp.bonds[b].t;
  }
  for (int i = threadIdx.x; i < a.nw; i += kThreads) bm[i] = 0u;
  if (threadIdx.x == 0) {
    const uint32_t b0 = L.item_blk[item];
    uint32_t b1 = L.item_blk[item + 1];
    if (b1 == uint32_t(L.nblk) || L.blk_off[b1] == uint32_t(k1)) b1 -= 1;
    s_b0 = b0;
    s_b1 = b1;
  }
  __syncthreads();
  const uint32_t b0 = s_b0, b1 = s_b1;

  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const int lane = threadIdx.x & 31;
  const int g = lane % G;
  const int group = threadIdx.x / G;
  constexpr int kGroups = kThreads / G;
  const int ncols = a.ncols, ld = a.ld, ncp = a.ncp;
  const int ctile = G * VEC;
  double dot_acc = 0.0;

  for (uint32_t blk = b0; blk <= b1; ++blk) {
    const int bs = int(L.blk_off[blk]), be = int(L.blk_off[blk + 1]);
    const uint32_t major = L.blk_major[blk];
    const int bsz = be - bs;
    const bool staged = int64_t(bsz) * ncp <= a.xs_cap;
    for (int q = threadIdx.x; q < bsz; q += kThreads) {
      const uint32_t d = L.minor[bs + q];
      atomicOr(&bm[d >> 5], 1u << (d & 31));
      if (q == 0 || (L.minor[bs + q - 1] >> 5) != (d >> 5)) pre[d >> 5] = uint16_t(q);
    }
    if (staged) {
      if (ncp == 1) {
        for (int q = threadIdx.x; q < bsz; q += kThreads)
          xs[q] = x[int64_t(PASS_A ? bs + q : int(L.perm[bs + q])) * ld];
      } else {
        for (int e = threadIdx.x; e < bsz * ncp; e += kThreads) {
          const int q = e / ncp, cc = e - q * ncp;
          const int64_t row = PASS_A ? int64_t(bs + q) : int64_t(L.perm[bs + q]);
          xs[e] = cc < ncols ? x[row * ld + cc] : T(0);
        }
      }
    }
    __syncthreads();
    const int lo = (int64_t(bs) > k0) ? bs : int(k0);
    const int hi = (int64_t(be) < k1) ? be : int(k1);
    const int rounds = (hi - lo + kGroups - 1) / kGroups;
    using C = ChunkOf<T, VEC>;
    for (int r = 0; r < rounds; ++r) {
      const int k = lo + r * kGroups + group;
      const bool live = k < hi;
      const uint32_t m = live ? L.minor[k] : 0u;
      for (int c0 = 0; c0 < ncols; c0 += ctile) {
        const int col = c0 + g * VEC;
        const int cvalid = ncols - col;
        Acc<T> acc[VEC];
#pragma unroll
        for (int c = 0; c < VEC; ++c) acc[c].zero();
        for (int bb = 0; bb < nbonds; bb += G) {
          const int b = bb + g;
          int q = -1;
          Coef<T> cf{T(0), T(0)};
          if (live && b < nbonds) {
            const uint32_t mk = s_mask[b];
            if (__popc(m & mk) == 1) {
              const uint32_t m2 = m ^ mk;
              const uint32_t wd = bm[m2 >> 5];
              const uint32_t bit = m2 & 31u;
              if ((wd >> bit) & 1u) {
                q = int(pre[m2 >> 5]) + __popc(wd & ((1u << bit) - 1u));
                cf = bond_coef<T>(s_thi, s_tlo, s_t64, b, __popc(m & s_betw[b]) & 1);
              }
            }
          }
#pragma unroll
          for (int s = 0; s < G; ++s) {
            const int qq = G == 1 ? q : __shfl_sync(0xffffffffu, q, s, G);
            const T ch = G == 1 ? cf.hi : __shfl_sync(0xffffffffu, cf.hi, s, G);
            const T cl = G == 1 ? cf.lo : __shfl_sync(0xffffffffu, cf.lo, s, G);
            if (qq >= 0 && cvalid > 0) {
              T xv[VEC];
              if (staged) {
                const T* p = xs + qq * ncp + col;
                if (VEC == 1 || cvalid >= VEC) {
#pragma unroll
                  for (int c = 0; c < VEC; ++c) xv[c] = p[c];
                } else {
#pragma unroll
                  for (int c = 0; c < VEC; ++c) xv[c] = c < cvalid ? p[c] : T(0);
                }
              } else {
                const int64_t row = PASS_A ? int64_t(bs + qq) : int64_t(L.perm[bs + qq]);
                C::load(x + row * ld + col, cvalid, xv);
              }
#pragma unroll
              for (int c = 0; c < VEC; ++c) acc[c].fma(ch, cl, xv[c]);
            }
          }
        }
        if (live && cvalid > 0) {
          T out[VEC];
          if (PASS_A) {
            const Coef<T> dc = diag_coef<T>(hp, major, m);
            T xv[VEC], yv[VEC];
            C::load(x + int64_t(k) * ld + col, cvalid, xv);
            C::load(y + int64_t(k) * ld + col, cvalid, yv);
#pragma unroll
            for (int c = 0; c < VEC; ++c) {
              acc[c].fma(dc.hi, dc.lo, xv[c]);
              out[c] = acc[c].value() + yv[c];
            }
            if (DOT) dot_acc += double(xv[0]) * double(out[0]);
            C::store(y + int64_t(k) * ld + col, cvalid, out);
          } else {
#pragma unroll
            for (int c = 0; c < VEC; ++c) out[c] = acc[c].value();
            C::store(y + int64_t(L.perm[k]) * ld + col, cvalid, out);
          }
        }
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < bsz; q += kThreads) bm[L.minor[bs + q] >> 5] = 0u;
    __syncthreads();
  }

  if (DOT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot_acc += __shfl_xor_sync(0xffffffffu, dot_acc, o);
    if (lane == 0) s_red[threadIdx.x >> 5] = dot_acc;
    __syncthreads();
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) sum += s_red[w];
      a.dot_partials[blockIdx.x] = sum;
      __threadfence();
      const unsigned t = atomicAdd(a.ticket, 1u);
      s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
      double sum = 0.0;
      for (int i = threadIdx.x; i < int(gridDim.x); i += kThreads) sum += __ldcg(a.dot_partials + i);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      __syncthreads();
      if (lane == 0) s_red[threadIdx.x >> 5] = sum;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) tot += s_red[w];
        *a.dot_out = tot;
        *a.ticket = 0u;
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Single-column variant of the bitmap kernel (the Lanczos case), one thread per
// state.  Shared memory holds, per block, a 2^n-bit bitmap of its minor words
// packed with per-word prefix counts (uint2: bits, block-local index of the
// first state in the word), so one 8-byte load answers "is m2 in the block"
// and "where".  Active hops are enumerated from partner classes: for class c,
// (m ^ P_c(m)) & first_c marks its active bonds (P_c = bit permutation taken
// from two byte tables); two classes form one 32-bit mask whose bits are
// taken two at a time, so each thread keeps two independent lookups in
// flight.  Without partner classes every bond is tested in turn.
template <typename T>
struct L1Smem {
  const uint2* bm;              // [nw] bits, first local index
  const T* xs;                  // staged x of the block
  const uint2* ptab;            // [groups][2][256] P contributions, four classes per entry
  const uint2* pflip;           // [n_pcls * 16] (flip, between) by class and first endpoint
  const float* dhi;
  const float* dlo;
  const double* d64;
};

template <typename T, bool STAGED, bool PASS_A>
__device__ __forceinline__ T l1_fetch(const HvArgs& a, const Layout& L, const L1Smem<T>& S, int bs, int q) {
  if (STAGED) return S.xs[q];
  const T* x = static_cast<const T*>(a.x);
  return __ldg(x + (PASS_A ? int64_t(bs + q) : int64_t(L.perm[bs + q])) * a.ld);
}

// block-local index of m2, or -1
__device__ __forceinline__ int l1_find(const uint2* bm, uint32_t m2) {
  const uint2 w = bm[m2 >> 5];
  const uint32_t sh = m2 & 31u;
  return ((w.x >> sh) & 1u) ? int(w.y) + __popc(w.x & ((1u << sh) - 1u)) : -1;
}

template <typename T, bool PASS_A, bool DOT, bool STAGED, bool PARTNER>
__device__ __forceinline__ void l1_state(const HvArgs& a, const HamParams& hp, const Layout& L,
                                         const L1Smem<T>& S, uint32_t major, int bs, int k, double& dot_acc) {
  T* __restrict__ y = static_cast<T*>(a.y);
  const uint32_t m = L.minor[k];
  Acc<T> acc;
  acc.zero();
  if (PARTNER) {
    const uint32_t mm = m | (m << 16);
    for (int g = 0; 4 * g < hp.n_pcls; ++g) {
      const uint2 t0 = S.ptab[g * 512 + (m & 255u)];
      const uint2 t1 = S.ptab[g * 512 + 256 + (m >> 8)];
      for (int h = 0; h < 2; ++h) {
        const int c = 4 * g + 2 * h;
        if (c >= hp.n_pcls) break;
        const bool pair = c + 1 < hp.n_pcls;
        const uint32_t pp = h ? (t0.y | t1.y) : (t0.x | t1.x);
        uint32_t act = (mm ^ pp) & (hp.pfirst[c] | (pair ? hp.pfirst[c + 1] << 16 : 0u));
        const uint2* fl = S.pflip + c * 16;   // bit position p -> class c + (p >> 4), site p & 15
        T s0 = T(0), s1 = T(0);
        while (act) {
          const int i1 = __ffs(act) - 1;
          act &= act - 1u;
          const bool two = act != 0u;
          const int i2 = two ? __ffs(act) - 1 : i1;
          act &= act - 1u;   // no-op when act == 0
          const uint2 f1 = fl[i1];
          const uint2 f2 = fl[i2];
          const int q1 = l1_find(S.bm, m ^ f1.x);
          const int q2 = two ? l1_find(S.bm, m ^ f2.x) : -1;
          if (q1 >= 0) {
            T xv = l1_fetch<T, STAGED, PASS_A>(a, L, S, bs, q1);
            if (__popc(m & f1.y) & 1u) xv = -xv;
            if (i1 >> 4) s1 += xv; else s0 += xv;
          }
          if (q2 >= 0) {
            T xv = l1_fetch<T, STAGED, PASS_A>(a, L, S, bs, q2);
            if (__popc(m & f2.y) & 1u) xv = -xv;
            if (i2 >> 4) s1 += xv; else s0 += xv;
          }
        }
        if (sizeof(T) == 4) {
          acc.fma(T(hp.pcls_hi[c]), T(hp.pcls_lo[c]), s0);
          if (pair) acc.fma(T(hp.pcls_hi[c + 1]), T(hp.pcls_lo[c + 1]), s1);
        } else {
          acc.fma(T(hp.pcls_t[c]), T(0), s0);
          if (pair) acc.fma(T(hp.pcls_t[c + 1]), T(0), s1);
        }
      }
    }
  } else {
    int b = 0;
    for (int c = 0; c < hp.n_class; ++c) {
      const int e = hp.cls_end[c];
      T s = T(0);
      for (; b < e; ++b) {
        const uint32_t mk = hp.bonds[b].mask;
        if (__popc(m & mk) != 1) continue;
        const int q = l1_find(S.bm, m ^ mk);
        if (q < 0) continue;
        T xv = l1_fetch<T, STAGED, PASS_A>(a, L, S, bs, q);
        s += (__popc(m & hp.bonds[b].between) & 1u) ? -xv : xv;
      }
      if (sizeof(T) == 4) acc.fma(T(hp.cls_hi[c]), T(hp.cls_lo[c]), s);
      else acc.fma(T(hp.cls_t[c]), T(0), s);
    }
  }
  if (PASS_A) {
    const T* x = static_cast<const T*>(a.x);
    const T xk = STAGED ? S.xs[k - bs] : __ldg(x + int64_t(k) * a.ld);
    const int nu = __popc(major & m);
    if (hp.uniform) {
      if (sizeof(T) == 4) acc.fma(T(S.dhi[nu]), T(S.dlo[nu]), xk);
      else acc.fma(T(S.d64[nu]), T(0), xk);
    } else {
      const Coef<T> dc = diag_coef<T>(hp, major, m);
      acc.fma(dc.hi, dc.lo, xk);
    }
    const T out = acc.value() + y[int64_t(k) * a.ld];
    y[int64_t(k) * a.ld] = out;
    if (DOT) dot_acc += double(xk) * double(out);
  } else {
    y[int64_t(L.perm[k]) * a.ld] = acc.value();
  }
}

template <typename T, bool PASS_A, bool DOT>
__global__ void __launch_bounds__(kThreads) hv_l1_kernel(const HvArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ uint32_t s_b0, s_b1;
  __shared__ double s_red[kThreads / 32];
  __shared__ float s_dhi[kMaxSites + 1], s_dlo[kMaxSites + 1];
  __shared__ double s_d64[kMaxSites + 1];
  uint2* s_pt = reinterpret_cast<uint2*>(s_dyn + a.off_pt);
  uint2* bm = reinterpret_cast<uint2*>(s_dyn + a.off_bm);
  T* xs = reinterpret_cast<T*>(s_dyn + a.off_xs);
  const bool use_p = hp.n_pcls > 0;

  const Layout& L = a.L;
  const int item = blockIdx.x;
  const int64_t k0 = int64_t(item) * kItem;
  const int64_t k1 = (k0 + kItem < L.n) ? k0 + kItem : L.n;
  for (int i = threadIdx.x; i < a.nw; i += kThreads) bm[i] = make_uint2(0u, 0u);
  if (use_p)   // P table groups followed by the (flip, between) table, contiguous in global memory
    for (int i = threadIdx.x; i < ((hp.n_pcls + 3) / 4) * 512 + hp.n_pcls * 16; i += kThreads) s_pt[i] = hp.ptab[i];
  if (threadIdx.x <= kMaxSites) {
    s_dhi[threadIdx.x] = hp.dtab_hi[threadIdx.x];
    s_dlo[threadIdx.x] = hp.dtab_lo[threadIdx.x];
    s_d64[threadIdx.x] = hp.dtab[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    const uint32_t b0 = L.item_blk[item];
    uint32_t b1 = L.item_blk[item + 1];
    if (b1 == uint32_t(L.nblk) || L.blk_off[b1] == uint32_t(k1)) b1 -= 1;
    s_b0 = b0;
    s_b1 = b1;
  }
  __syncthreads();
  const uint32_t b0 = s_b0, b1 = s_b1;
  const T* __restrict__ x = static_cast<const T*>(a.x);
  L1Smem<T> S{bm, xs, s_pt, s_pt + ((hp.n_pcls + 3) / 4) * 512, s_dhi, s_dlo, s_d64};
  double dot_acc = 0.0;

  for (uint32_t blk = b0; blk <= b1; ++blk) {
    const int bs = int(L.blk_off[blk]), be = int(L.blk_off[blk + 1]);
    const uint32_t major = L.blk_major[blk];
    const int bsz = be - bs;
    const bool staged = bsz <= a.xs_cap;
    // build: loads of four states are issued before any of them is used
    for (int q0 = threadIdx.x; q0 < bsz; q0 += 4 * kThreads) {
      uint32_t d[4], dp[4];
      T xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * kThreads;
        d[u] = q < bsz ? __ldg(L.minor + bs + q) : 0u;
        dp[u] = (q < bsz && q > 0) ? __ldg(L.minor + bs + q - 1) : 0xFFFFFFFFu;
      }
      if (staged) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u * kThreads;
          xv[u] = q < bsz ? __ldg(x + (PASS_A ? int64_t(bs + q) : int64_t(__ldg(L.perm + bs + q))) * a.ld) : T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * kThreads;
        if (q < bsz) {
          atomicOr(&bm[d[u] >> 5].x, 1u << (d[u] & 31));
          if (q == 0 || (dp[u] >> 5) != (d[u] >> 5)) bm[d[u] >> 5].y = uint32_t(q);
          if (staged) xs[q] = xv[u];
        }
      }
    }
    __syncthreads();
    const int lo = (int64_t(bs) > k0) ? bs : int(k0);
    const int hi = (int64_t(be) < k1) ? be : int(k1);
    if (use_p) {
      if (staged) {
        for (int k = lo + threadIdx.x; k < hi; k += kThreads)
          l1_state<T, PASS_A, DOT, true, true>(a, hp, L, S, major, bs, k, dot_acc);
      } else {
        for (int k = lo + threadIdx.x; k < hi; k += kThreads)
          l1_state<T, PASS_A, DOT, false, true>(a, hp, L, S, major, bs, k, dot_acc);
      }
    } else if (staged) {
      for (int k = lo + threadIdx.x; k < hi; k += kThreads)
        l1_state<T, PASS_A, DOT, true, false>(a, hp, L, S, major, bs, k, dot_acc);
    } else {
      for (int k = lo + threadIdx.x; k < hi; k += kThreads)
        l1_state<T, PASS_A, DOT, false, false>(a, hp, L, S, major, bs, k, dot_acc);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < bsz; q += kThreads) bm[L.minor[bs + q] >> 5].x = 0u;
    __syncthreads();
  }

  if (DOT) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot_acc += __shfl_xor_sync(0xffffffffu, dot_acc, o);
    if (lane == 0) s_red[threadIdx.x >> 5] = dot_acc;
    __syncthreads();
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) sum += s_red[w];
      a.dot_partials[blockIdx.x] = sum;
      __threadfence();
      const unsigned t = atomicAdd(a.ticket, 1u);
      s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
      double sum = 0.0;
      for (int i = threadIdx.x; i < int(gridDim.x); i += kThreads) sum += __ldcg(a.dot_partials + i);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      __syncthreads();
      if (lane == 0) s_red[threadIdx.x >> 5] = sum;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) tot += s_red[w];
        *a.dot_out = tot;
        *a.ticket = 0u;
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Multi-column variant (H~V, band Lanczos).  Rounds of 256 states; in phase
// 1 one thread per state enumerates its active hops from the partner classes
// and looks them up once, writing each found target as a 2-byte record
// (block-local index | sign << 14 | class-half << 15) into one shared list
// per state, in class-pair order, with the list's end after each pair (at
// most kLcCap records; a state with more is flagged and its hops are found
// again by its lanes in phase 2).  In phase 2 groups of G lanes read the
// lists of their states and gather and sum the VEC columns each lane owns
// (from staged block rows when they fit), four rows in flight.  The compact
// lists keep a CTA at ~52 KiB of shared memory, four CTAs per SM.
template <typename T, int VEC, int G, bool PASS_A>
__global__ void __launch_bounds__(kThreads) hv_lc_kernel(const HvArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ uint32_t s_b0, s_b1;
  __shared__ float s_dhi[kMaxSites + 1], s_dlo[kMaxSites + 1];
  __shared__ double s_d64[kMaxSites + 1];
  uint2* s_pt = reinterpret_cast<uint2*>(s_dyn + a.off_pt);
  uint2* bm = reinterpret_cast<uint2*>(s_dyn + a.off_bm);
  T* xs = reinterpret_cast<T*>(s_dyn + a.off_xs);
  uint16_t* lists = reinterpret_cast<uint16_t*>(s_dyn + a.off_list);   // [256][kLcCap]
  uint8_t* cnts = reinterpret_cast<uint8_t*>(s_dyn + a.off_cnt);        // [256][npairs] list ends
  uint8_t* ovf = cnts + kThreads * ((hp.n_pcls + 1) / 2);                // [256] list overflowed
  const Layout& L = a.L;
  const int item = blockIdx.x;
  const int64_t k0 = int64_t(item) * kItem;
  const int64_t k1 = (k0 + kItem < L.n) ? k0 + kItem : L.n;
  const int ng = (hp.n_pcls + 3) / 4;
  const int npairs = (hp.n_pcls + 1) / 2;
  for (int i = threadIdx.x; i < a.nw; i += kThreads) bm[i] = make_uint2(0u, 0u);
  for (int i = threadIdx.x; i < ng * 512 + hp.n_pcls * 16; i += kThreads) s_pt[i] = hp.ptab[i];
  if (threadIdx.x <= kMaxSites) {
    s_dhi[threadIdx.x] = hp.dtab_hi[threadIdx.x];
    s_dlo[threadIdx.x] = hp.dtab_lo[threadIdx.x];
    s_d64[threadIdx.x] = hp.dtab[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    const uint32_t b0 = L.item_blk[item];
    uint32_t b1 = L.item_blk[item + 1];
    if (b1 == uint32_t(L.nblk) || L.blk_off[b1] == uint32_t(k1)) b1 -= 1;
    s_b0 = b0;
    s_b1 = b1;
  }
  __syncthreads();
  const uint2* ptab = s_pt;
  const uint2* pflip = s_pt + ng * 512;
  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const int g = threadIdx.x % G;
  const int group = threadIdx.x / G;
  constexpr int kGroups = kThreads / G;
  const int ncols = a.ncols, ld = a.ld, ncp = a.ncp;
  const int col = g * VEC;
  const int cvalid = ncols - col;
  using C = ChunkOf<T, VEC>;
  uint16_t* mylist = lists + threadIdx.x * kLcCap;
  uint8_t* mycnt = cnts + threadIdx.x * npairs;

  for (uint32_t blk = s_b0; blk <= s_b1; ++blk) {
    const int bs = int(L.blk_off[blk]), be = int(L.blk_off[blk + 1]);
    const uint32_t major = L.blk_major[blk];
    const int bsz = be - bs;
    const bool staged = int64_t(bsz) * ncp <= a.xs_cap;
    for (int q = threadIdx.x; q < bsz; q += kThreads) {
      const uint32_t d = L.minor[bs + q];
      atomicOr(&bm[d >> 5].x, 1u << (d & 31));
      if (q == 0 || (L.minor[bs + q - 1] >> 5) != (d >> 5)) bm[d >> 5].y = uint32_t(q);
    }
    if (staged && col < ncp) {
      for (int q = group; q < bsz; q += kGroups) {
        const int64_t row = PASS_A ? int64_t(bs + q) : int64_t(L.perm[bs + q]);
        T v[VEC];
        C::load(x + row * ld + col, cvalid, v);
#pragma unroll
        for (int u = 0; u < VEC; ++u) xs[q * ncp + col + u] = v[u];
      }
    }
    __syncthreads();
    const int lo = (int64_t(bs) > k0) ? bs : int(k0);
    const int hi = (int64_t(be) < k1) ? be : int(k1);
    for (int r0 = lo; r0 < hi; r0 += kThreads) {
      // phase 1: lookups, one thread per state
      {
        const int k = r0 + threadIdx.x;
        int nf = 0;
        if (k < hi) {
          const uint32_t m = L.minor[k];
          const uint32_t mm = m | (m << 16);
          for (int gi = 0; gi < ng; ++gi) {
            const uint2 t0 = ptab[gi * 512 + (m & 255u)];
            const uint2 t1 = ptab[gi * 512 + 256 + (m >> 8)];
            for (int h = 0; h < 2; ++h) {
              const int c = 4 * gi + 2 * h;
              if (c >= hp.n_pcls) break;
              const bool pair = c + 1 < hp.n_pcls;
              const uint32_t pp = h ? (t0.y | t1.y) : (t0.x | t1.x);
              uint32_t act = (mm ^ pp) & (hp.pfirst[c] | (pair ? hp.pfirst[c + 1] << 16 : 0u));
              const uint2* fl = pflip + c * 16;
              while (act) {
                const int i1 = __ffs(act) - 1;
                act &= act - 1u;
                const uint2 f1 = fl[i1];
                const int q1 = l1_find(bm, m ^ f1.x);
                if (q1 >= 0) {
                  if (nf < kLcCap)
                    mylist[nf] = uint16_t(q1 | ((__popc(m & f1.y) & 1u) << 14) | ((i1 >> 4) << 15));
                  ++nf;
                }
              }
              mycnt[c >> 1] = uint8_t(nf < kLcCap ? nf : kLcCap);
            }
          }
        } else {
          for (int pi = 0; pi < npairs; ++pi) mycnt[pi] = 0;
        }
        ovf[threadIdx.x] = nf > kLcCap ? 1 : 0;
      }
      __syncthreads();
      // phase 2: gathers, G lanes per state
      const int ns = (hi - r0 < kThreads) ? hi - r0 : kThreads;
      for (int t = group; t < ns; t += kGroups) {
        const int k = r0 + t;
        const uint16_t* lt = lists + t * kLcCap;
        const uint8_t* ct = cnts + t * npairs;
        const bool over = ovf[t] != 0;
        const uint32_t mk = over ? L.minor[k] : 0u;
        const uint32_t mmk = mk | (mk << 16);
        Acc<T> acc[VEC];
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[u].zero();
        for (int pi = 0; pi < npairs; ++pi) {
          const int c = 2 * pi;
          const bool pair = c + 1 < hp.n_pcls;
          T s0[VEC], s1[VEC];
#pragma unroll
          for (int u = 0; u < VEC; ++u) s0[u] = s1[u] = T(0);
          const int jb = pi ? int(ct[pi - 1]) : 0;
          const int nf = (cvalid > 0 && !over) ? int(ct[pi]) : 0;
          if (over && cvalid > 0) {
            // the state's list overflowed: find this pair's hops again, in
            // the order phase 1 uses
            const int gi = c >> 2, h = (c >> 1) & 1;
            const uint2 t0 = ptab[gi * 512 + (mk & 255u)];
            const uint2 t1 = ptab[gi * 512 + 256 + (mk >> 8)];
            const uint32_t pp = h ? (t0.y | t1.y) : (t0.x | t1.x);
            uint32_t act = (mmk ^ pp) & (hp.pfirst[c] | (pair ? hp.pfirst[c + 1] << 16 : 0u));
            const uint2* fl = pflip + c * 16;
            while (act) {
              const int i1 = __ffs(act) - 1;
              act &= act - 1u;
              const uint2 f1 = fl[i1];
              const int q = l1_find(bm, mk ^ f1.x);
              if (q < 0) continue;
              T xv[VEC];
              if (staged) {
#pragma unroll
                for (int u = 0; u < VEC; ++u) xv[u] = xs[q * ncp + col + u];
              } else {
                const int64_t row = PASS_A ? int64_t(bs + q) : int64_t(L.perm[bs + q]);
                C::load(x + row * ld + col, cvalid, xv);
              }
              const bool neg = __popc(mk & f1.y) & 1u;
              if (i1 >> 4) {
#pragma unroll
                for (int u = 0; u < VEC; ++u) s1[u] += neg ? -xv[u] : xv[u];
              } else {
#pragma unroll
                for (int u = 0; u < VEC; ++u) s0[u] += neg ? -xv[u] : xv[u];
              }
            }
          }
          // rows of up to four hits are loaded before any is added (four
          // independent loads in flight); the sums keep the list order
          for (int j0 = jb; j0 < nf; j0 += 4) {
            uint32_t e[4];
            T xv[4][VEC];
#pragma unroll
            for (int h = 0; h < 4; ++h) e[h] = j0 + h < nf ? uint32_t(lt[j0 + h]) : 0u;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              if (j0 + h >= nf) break;
              const int q = int(e[h] & 0x3FFFu);
              if (staged) {
#pragma unroll
                for (int u = 0; u < VEC; ++u) xv[h][u] = xs[q * ncp + col + u];
              } else {
                const int64_t row = PASS_A ? int64_t(bs + q) : int64_t(L.perm[bs + q]);
                C::load(x + row * ld + col, cvalid, xv[h]);
              }
            }
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              if (j0 + h >= nf) break;
              const bool neg = e[h] & 0x4000u;
              if (e[h] & 0x8000u) {
#pragma unroll
                for (int u = 0; u < VEC; ++u) s1[u] += neg ? -xv[h][u] : xv[h][u];
              } else {
#pragma unroll
                for (int u = 0; u < VEC; ++u) s0[u] += neg ? -xv[h][u] : xv[h][u];
              }
            }
          }
#pragma unroll
          for (int u = 0; u < VEC; ++u) {
            if (sizeof(T) == 4) {
              acc[u].fma(T(hp.pcls_hi[c]), T(hp.pcls_lo[c]), s0[u]);
              if (pair) acc[u].fma(T(hp.pcls_hi[c + 1]), T(hp.pcls_lo[c + 1]), s1[u]);
            } else {
              acc[u].fma(T(hp.pcls_t[c]), T(0), s0[u]);
              if (pair) acc[u].fma(T(hp.pcls_t[c + 1]), T(0), s1[u]);
            }
          }
        }
        if (cvalid > 0) {
          T out[VEC];
          if (PASS_A) {
            const uint32_t m = L.minor[k];
            T xv[VEC], yv[VEC];
            if (staged) {
#pragma unroll
              for (int u = 0; u < VEC; ++u) xv[u] = xs[(k - bs) * ncp + col + u];
            } else {
              C::load(x + int64_t(k) * ld + col, cvalid, xv);
            }
            C::load(y + int64_t(k) * ld + col, cvalid, yv);
            const int nu = __popc(major & m);
            Coef<T> dc;
            if (hp.uniform) {
              dc.hi = sizeof(T) == 4 ? T(s_dhi[nu]) : T(s_d64[nu]);
              dc.lo = sizeof(T) == 4 ? T(s_dlo[nu]) : T(0);
            } else {
              dc = diag_coef<T>(hp, major, m);
            }
#pragma unroll
            for (int u = 0; u < VEC; ++u) {
              acc[u].fma(dc.hi, dc.lo, xv[u]);
              out[u] = acc[u].value() + yv[u];
            }
            C::store(y + int64_t(k) * ld + col, cvalid, out);
          } else {
#pragma unroll
            for (int u = 0; u < VEC; ++u) out[u] = acc[u].value();
            C::store(y + int64_t(L.perm[k]) * ld + col, cvalid, out);
          }
        }
      }
      __syncthreads();
    }
    for (int q = threadIdx.x; q < bsz; q += kThreads) bm[L.minor[bs + q] >> 5].x = 0u;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// Plain path: one thread per state, both spins, binary search over the whole
// sorted basis in global memory.  Kept as the simple reference GPU path.
template <typename T>
__global__ void hv_plain_kernel(const uint64_t* __restrict__ words, int64_t n, const T* __restrict__ x,
                                T* __restrict__ y, int ncols, int ld, const HamParams hp) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int ns = hp.n_sites;
  const uint64_t w = words[k];
  const uint64_t half = ns == 32 ? 0xFFFFFFFFull : ((1ull << ns) - 1);
  const uint32_t up = uint32_t(w >> ns), dn = uint32_t(w & half);
  const double d = diag_f64(hp, up, dn);
  for (int c = 0; c < ncols; ++c) {
    double acc = d * double(x[k * ld + c]);
    for (int spin = 0; spin < 2; ++spin) {
      const uint32_t ws = spin == 0 ? up : dn;
      const int shift = spin == 0 ? ns : 0;
      for (int b = 0; b < hp.n_bonds; ++b) {
        const uint32_t mk = hp.bonds[b].mask;
        if (__popc(ws & mk) != 1) continue;
        const uint64_t w2 = w ^ (uint64_t(mk) << shift);
        int64_t lo = 0, len = n;
        while (len > 1) {
          const int64_t h = len >> 1;
          if (words[lo + h] <= w2) lo += h;
          len -= h;
        }
        if (words[lo] != w2) continue;
        const double t = (__popc(ws & hp.bonds[b].between) & 1) ? -hp.bonds[b].t : hp.bonds[b].t;
        acc += t * double(x[lo * ld + c]);
      }
    }
    y[k * ld + c] = T(acc);
  }
}

__global__ void diag_kernel(const uint64_t* __restrict__ words, int64_t n, double* out, const HamParams hp) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int ns = hp.n_sites;
  const uint64_t w = words[k];
  const uint64_t half = ns == 32 ? 0xFFFFFFFFull : ((1ull << ns) - 1);
  out[k] = diag_f64(hp, uint32_t(w >> ns), uint32_t(w & half));
}

// Connection dump, same hop enumeration, sign and in-block search as the
// block kernels, one thread per state of a layout.  mode 0: cnt[row] +=
// connections of this pass; mode 1: write triples at off[row] + (mode-1 base).
template <bool PASS_A>
__global__ void conn_kernel(const Layout L, const HamParams hp, uint32_t* cnt, const uint64_t* off,
                            const uint32_t* cnt_first, int64_t* rows, int64_t* cols, double* vals, int write) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= L.n) return;
  // block of k: binary search over blk_off
  int64_t lo = 0, len = L.nblk;
  while (len > 1) {
    const int64_t h = len >> 1;
    if (L.blk_off[lo + h] <= uint32_t(k)) lo += h;
    len -= h;
  }
  const int bbase = int(L.blk_off[lo]), bend = int(L.blk_off[lo + 1]);
  const uint32_t m = L.minor[k];
  const int64_t row = PASS_A ? k : int64_t(L.perm[k]);
  int64_t w = 0;
  if (write) w = int64_t(off[row]) + (PASS_A ? int64_t(cnt_first[row]) : 0);
  uint32_t c = 0;
  for (int b = 0; b < hp.n_bonds; ++b) {
    const uint32_t mk = hp.bonds[b].mask;
    if (__popc(m & mk) != 1) continue;
    const int q = find_sorted(L.minor, bbase, bend, m ^ mk);
    if (q < 0) continue;
    if (write) {
      rows[w] = row;
      cols[w] = PASS_A ? int64_t(q) : int64_t(L.perm[q]);
      vals[w] = (__popc(m & hp.bonds[b].between) & 1) ? -hp.bonds[b].t : hp.bonds[b].t;
      ++w;
    }
    ++c;
  }
  if (!write) cnt[row] = c;
}

__global__ void sum_counts_kernel(const uint32_t* a, const uint32_t* b, int64_t n, unsigned long long* out,
                                  uint64_t* excl /*nullable*/) {
  // single-block running sum (n is at most ~1e8 and this runs once per basis)
  __shared__ unsigned long long s_part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t lo = t * chunk, hi = (lo + chunk < n ? lo + chunk : n);
  unsigned long long s = 0;
  for (int64_t i = lo; i < hi; ++i) s += uint64_t(a[i]) + uint64_t(b[i]);
  s_part[t] = s;
  __syncthreads();
  if (t == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < int(blockDim.x); ++i) {
      const unsigned long long v = s_part[i];
      s_part[i] = run;
      run += v;
    }
    *out = run;
  }
  __syncthreads();
  if (excl) {
    unsigned long long run = s_part[t];
    for (int64_t i = lo; i < hi; ++i) {
      excl[i] = run;
      run += uint64_t(a[i]) + uint64_t(b[i]);
    }
  }
}

int grid_of(int64_t n, int t) { return int((n + t - 1) / t); }

template <typename T, int VEC, int G>
cudaError_t launch_pair(mcd_ctx* c, const void* x, void* y, int ncols, int ld, double* partials,
                        unsigned int* ticket, double* dot_out) {
  HvArgs a;
  a.x = x;
  a.y = y;
  a.ncols = ncols;
  a.ld = ld;
  a.n_sites = c->n;
  a.dot_partials = partials;
  a.ticket = ticket;
  a.dot_out = dot_out;
  const bool bitmap = c->n <= kBitmapMaxSites && c->hv_algo == 0;
  size_t smem = kStageWords * sizeof(uint32_t);
  if (bitmap) {
    a.nbp = (c->hp->n_bonds + 3) & ~3;
    a.nw = c->n >= 5 ? (1 << (c->n - 5)) : 1;
    a.off_bm = 24 * a.nbp;
    a.off_pre = a.off_bm + 4 * a.nw;
    a.off_xs = (a.off_pre + 2 * a.nw + 15) & ~15;
    a.ncp = ((ncols + VEC - 1) / VEC) * VEC;
    a.xs_cap = int(kStageXBytes / sizeof(T));
    smem = size_t(a.off_xs) + kStageXBytes;
  }
  static std::atomic<int> configured_smem{-1};   // per instantiation; one device per process in practice
  if (configured_smem < int(smem)) {
    if (bitmap) {
      cudaFuncSetAttribute(hv_bitmap_kernel<T, VEC, G, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      cudaFuncSetAttribute(hv_bitmap_kernel<T, VEC, G, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      cudaFuncSetAttribute(hv_bitmap_kernel<T, VEC, G, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    }
    const int sm2 = kStageWords * sizeof(uint32_t);
    cudaFuncSetAttribute(hv_block_kernel<T, VEC, G, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
    cudaFuncSetAttribute(hv_block_kernel<T, VEC, G, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
    cudaFuncSetAttribute(hv_block_kernel<T, VEC, G, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
    configured_smem = int(smem);
  }
  const bool l1 = bitmap && G == 1 && VEC == 1 && ncols == 1 && (c->hp->n_class > 0 || c->hp->n_bonds == 0);
  if (l1) {
    // layout: [ptab: groups x 512 uint2][bm: nw uint2][xs]
    const int ng = (c->hp->n_pcls + 3) / 4;
    a.off_pt = 0;
    a.off_bm = (ng * 512 + c->hp->n_pcls * 16) * 8;
    a.off_xs = (a.off_bm + 8 * a.nw + 15) & ~15;
    smem = size_t(a.off_xs) + kStageX1Bytes;
    a.xs_cap = int(kStageX1Bytes / sizeof(T));
    static std::atomic<int> configured_l1{-1};
    if (configured_l1 < int(smem)) {
      cudaFuncSetAttribute(hv_l1_kernel<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      cudaFuncSetAttribute(hv_l1_kernel<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      cudaFuncSetAttribute(hv_l1_kernel<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      configured_l1 = int(smem);
    }
    a.L = c->idx.B;
    timing_begin(c, 0);
    hv_l1_kernel<T, false, false><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    a.L = c->idx.A;
    timing_begin(c, 1);
    if (partials)
      hv_l1_kernel<T, true, true><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
    else
      hv_l1_kernel<T, true, false><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    return cudaGetLastError();
  }
  const bool lc = bitmap && !l1 && c->hp->n_pcls > 0 && c->hp->n_pcls <= 8 && !partials && ncols <= G * VEC;
  if (lc) {
    // layout: [ptab + flips][bm: nw uint2][lists: 256 x kLcCap u16][list ends: 256 x npairs]
    //         [overflow flags: 256][xs]
    const int ngp = (c->hp->n_pcls + 3) / 4;
    const int npairs = (c->hp->n_pcls + 1) / 2;
    a.off_pt = 0;
    a.off_bm = (ngp * 512 + c->hp->n_pcls * 16) * 8;
    a.off_list = a.off_bm + 8 * a.nw;
    a.off_cnt = a.off_list + kThreads * kLcCap * 2;
    a.off_xs = (a.off_cnt + kThreads * npairs + kThreads + 15) & ~15;
    // staging area: what is left of ~52 KiB (four CTAs per SM), at least 1 KiB
    const int xs_bytes = std::max(1024, kStageXcBytes - a.off_xs) & ~15;
    smem = size_t(a.off_xs) + xs_bytes;
    a.xs_cap = int(xs_bytes / sizeof(T));
    static std::atomic<int> configured_lc{-1};
    if (configured_lc < int(smem)) {
      cudaFuncSetAttribute(hv_lc_kernel<T, VEC, G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      cudaFuncSetAttribute(hv_lc_kernel<T, VEC, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      configured_lc = int(smem);
    }
    a.L = c->idx.B;
    timing_begin(c, 0);
    hv_lc_kernel<T, VEC, G, false><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    a.L = c->idx.A;
    timing_begin(c, 1);
    hv_lc_kernel<T, VEC, G, true><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    return cudaGetLastError();
  }
  a.L = c->idx.B;
  timing_begin(c, 0);
  if (bitmap)
    hv_bitmap_kernel<T, VEC, G, false, false><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
  else
    hv_block_kernel<T, VEC, G, false, false><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
  MCD_LAUNCHED(c);
  timing_end(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  a.L = c->idx.A;
  timing_begin(c, 1);
  if (bitmap) {
    if (partials)
      hv_bitmap_kernel<T, VEC, G, true, true><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
    else
      hv_bitmap_kernel<T, VEC, G, true, false><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
  } else {
    if (partials)
      hv_block_kernel<T, VEC, G, true, true><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
    else
      hv_block_kernel<T, VEC, G, true, false><<<int(a.L.n_items), kThreads, smem, c->stream>>>(a, *c->hp);
  }
  MCD_LAUNCHED(c);
  timing_end(c);
  return cudaGetLastError();
}

template <typename T, int VEC>
cudaError_t dispatch_g(mcd_ctx* c, const void* x, void* y, int ncols, int ld, double* partials,
                       unsigned int* ticket, double* dot_out) {
  const int chunks = (ncols + VEC - 1) / VEC;
  if (chunks <= 1) return launch_pair<T, VEC, 1>(c, x, y, ncols, ld, partials, ticket, dot_out);
  if (chunks <= 2) return launch_pair<T, VEC, 2>(c, x, y, ncols, ld, partials, ticket, dot_out);
  if (chunks <= 4) return launch_pair<T, VEC, 4>(c, x, y, ncols, ld, partials, ticket, dot_out);
  if (chunks <= 8) return launch_pair<T, VEC, 8>(c, x, y, ncols, ld, partials, ticket, dot_out);
  if (chunks <= 16) return launch_pair<T, VEC, 16>(c, x, y, ncols, ld, partials, ticket, dot_out);
  return launch_pair<T, VEC, 32>(c, x, y, ncols, ld, partials, ticket, dot_out);
}

}  // namespace

// ---- timing ---------------------------------------------------------------------
void timing_begin(mcd_ctx* c, int cls) {
  if (!c->timing || !c->tm) return;
  Timing& t = *c->tm;
  if (t.n_ev >= 1024) timing_collect(c);
  const int i = t.n_ev;
  t.cls[i] = cls;
  cudaEventRecord(t.ev[2 * i], c->stream);
}
void timing_end(mcd_ctx* c) {
  if (!c->timing || !c->tm) return;
  Timing& t = *c->tm;
  cudaEventRecord(t.ev[2 * t.n_ev + 1], c->stream);
  ++t.n_ev;
}
void timing_collect(mcd_ctx* c) {
  if (!c->tm) return;
  Timing& t = *c->tm;
  if (t.n_ev == 0) return;
  cudaEventSynchronize(t.ev[2 * t.n_ev - 1]);
  for (int i = 0; i < t.n_ev; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.ev[2 * i], t.ev[2 * i + 1]) == cudaSuccess) {
      t.ms[t.cls[i]] += ms;
      t.count[t.cls[i]] += 1;
    }
  }
  t.n_ev = 0;
}

int hv_dot_ctas(mcd_ctx* c, int, int) { return int(c->idx.A.n_items); }

int hv_apply(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, double* dot_partials,
             int dot_slot) {
  (void)dot_slot;
  cudaError_t e = cudaSuccess;
  if (c->hv_algo == 1) {
    const int T = 256;
    timing_begin(c, 3);
    if (dtype == MCD_F64)
      hv_plain_kernel<double><<<grid_of(c->idx.n, T), T, 0, c->stream>>>(
          c->idx.words, c->idx.n, static_cast<const double*>(x), static_cast<double*>(y), ncols, ld, *c->hp);
    else
      hv_plain_kernel<float><<<grid_of(c->idx.n, T), T, 0, c->stream>>>(
          c->idx.words, c->idx.n, static_cast<const float*>(x), static_cast<float*>(y), ncols, ld, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "plain H*v launch");
    // the block kernels fuse <x, H x> into their last pass; here it is separate
    if (dot_partials) return vec_dot(c, x, y, c->idx.n, dtype, c->lw.scal + dot_slot);
    return MCD_OK;
  }
  unsigned int* ticket = nullptr;
  double* dot_out = nullptr;
  if (dot_partials) {
    ticket = c->lw.ticket;
    dot_out = c->lw.scal + dot_slot;
  }
  if (c->hv_algo == 0 && c->hv_cache != 1) {
    bool used = false;
    const int st = cache_apply(c, x, y, ncols, ld, dtype, dot_partials, dot_partials ? c->lw.max_ctas : 0, ticket,
                               dot_out, &used);
    if (st != MCD_OK || used) return st;
  }
  if (hash_eligible(c))
    return hash_apply(c, x, y, ncols, ld, dtype, dot_partials, dot_partials ? c->lw.max_ctas : 0, ticket, dot_out);
  const bool vec_ok = [&] {
    const size_t es = dtype == MCD_F64 ? 8 : 4;
    const int vec = dtype == MCD_F64 ? 2 : 4;
    return ncols > 1 && ld % vec == 0 && (reinterpret_cast<uintptr_t>(x) % 16 == 0) &&
           (reinterpret_cast<uintptr_t>(y) % 16 == 0) && es > 0;
  }();
  if (dtype == MCD_F64) {
    e = vec_ok ? dispatch_g<double, 2>(c, x, y, ncols, ld, dot_partials, ticket, dot_out)
               : dispatch_g<double, 1>(c, x, y, ncols, ld, dot_partials, ticket, dot_out);
  } else {
    e = vec_ok ? dispatch_g<float, 4>(c, x, y, ncols, ld, dot_partials, ticket, dot_out)
               : dispatch_g<float, 1>(c, x, y, ncols, ld, dot_partials, ticket, dot_out);
  }
  return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "H*v launch");
}

int hv_diagonal(mcd_ctx* c, double* out) {
  const int T = 256;
  diag_kernel<<<grid_of(c->idx.n, T), T, 0, c->stream>>>(c->idx.words, c->idx.n, out, *c->hp);
  MCD_LAUNCHED(c);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "diagonal");
}

int hv_connections(mcd_ctx* c, int64_t* rows, int64_t* cols, double* vals, int64_t cap, int64_t* nnz) {
  const int64_t n = c->idx.n;
  const int T = 256;
  cudaStream_t s = c->stream;
  uint32_t *ca = nullptr, *cb = nullptr;
  uint64_t* off = nullptr;
  unsigned long long* tot = nullptr;
  cudaError_t e = cudaMallocAsync(&ca, n * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&cb, n * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&off, n * 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&tot, 8, s);
  unsigned long long htot = 0;
  if (e == cudaSuccess) {
    conn_kernel<false><<<grid_of(n, T), T, 0, s>>>(c->idx.B, *c->hp, cb, nullptr, nullptr, nullptr, nullptr,
                                                   nullptr, 0);
    MCD_LAUNCHED(c);
    conn_kernel<true><<<grid_of(n, T), T, 0, s>>>(c->idx.A, *c->hp, ca, nullptr, nullptr, nullptr, nullptr,
                                                  nullptr, 0);
    MCD_LAUNCHED(c);
    sum_counts_kernel<<<1, 1024, 0, s>>>(cb, ca, n, tot, rows ? off : nullptr);
    MCD_LAUNCHED(c);
    e = cudaMemcpyAsync(&htot, tot, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess && rows) {
    if (int64_t(htot) > cap) {
      cudaFreeAsync(ca, s); cudaFreeAsync(cb, s); cudaFreeAsync(off, s); cudaFreeAsync(tot, s);
      *nnz = int64_t(htot);
      return fail(c, MCD_E_INVALID, "connections: capacity too small");
    }
    conn_kernel<false><<<grid_of(n, T), T, 0, s>>>(c->idx.B, *c->hp, nullptr, off, nullptr, rows, cols, vals, 1);
    MCD_LAUNCHED(c);
    conn_kernel<true><<<grid_of(n, T), T, 0, s>>>(c->idx.A, *c->hp, nullptr, off, cb, rows, cols, vals, 1);
    MCD_LAUNCHED(c);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFreeAsync(ca, s); cudaFreeAsync(cb, s); cudaFreeAsync(off, s); cudaFreeAsync(tot, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "connections");
  *nnz = int64_t(htot);
  c->idx.nnz = int64_t(htot);
  return MCD_OK;
}

}  // namespace mcd
