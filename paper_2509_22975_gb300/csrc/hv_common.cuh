// Device helpers shared by the H~v kernels (hv.cu, hv_hash.cu): launch
// arguments, vectorised row chunks, fp32 accumulation with fp64 coefficients
// split into two floats, the sorted-array search and the diagonal of Eq. (1).
#pragma once

#include <type_traits>

#include "mcd_internal.h"

namespace mcd {
namespace {

struct HvArgs {
  const void* x;
  void* y;
  int ncols;
  int ld;
  Layout L;
  int n_sites;
  double* dot_partials;   // pass A, single column: per-CTA sum x[k] y[k]
  unsigned int* ticket;
  double* dot_out;
  // bitmap kernel: dynamic shared-memory carve-up (bytes) and sizes
  int nbp;                // bonds rounded up to a multiple of 4
  int nw;                 // bitmap words = max(1, 2^n_sites / 32)
  int off_bm, off_pre, off_xs;
  int xs_cap;             // elements of T that fit in the x staging area
  int off_pt;             // single-column kernel: partner table
  int off_list, off_cnt;  // multi-column kernel: per-state connection lists
  int ncp;                // staged row stride: ncols rounded up to VEC
  // hash kernel: work items, per-block tables, shared table size
  const HItem* items;
  int n_hitems;
  const uint32_t* htab;
  const uint32_t* hflt;
  int hlog2;              // log2 of the shared table slots
  int flog2;              // log2 of the shared filter bits
  int hcap;               // states per work item
};

template <typename T, int VEC>
struct Chunk;
template <>
struct Chunk<float, 4> {
  static __device__ __forceinline__ void load(const float* p, int cvalid, float* v) {
    if (cvalid >= 4) {
      float4 q = __ldg(reinterpret_cast<const float4*>(p));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = c < cvalid ? __ldg(p + c) : 0.f;
    }
  }
  static __device__ __forceinline__ void store(float* p, int cvalid, const float* v) {
    if (cvalid >= 4) {
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < cvalid) p[c] = v[c];
    }
  }
};
template <>
struct Chunk<double, 2> {
  static __device__ __forceinline__ void load(const double* p, int cvalid, double* v) {
    if (cvalid >= 2) {
      double2 q = __ldg(reinterpret_cast<const double2*>(p));
      v[0] = q.x; v[1] = q.y;
    } else {
      v[0] = cvalid > 0 ? __ldg(p) : 0.0;
      v[1] = 0.0;
    }
  }
  static __device__ __forceinline__ void store(double* p, int cvalid, const double* v) {
    if (cvalid >= 2)
      *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    else if (cvalid > 0)
      p[0] = v[0];
  }
};
template <typename T>
struct Chunk1 {
  static __device__ __forceinline__ void load(const T* p, int cvalid, T* v) { v[0] = cvalid > 0 ? __ldg(p) : T(0); }
  static __device__ __forceinline__ void store(T* p, int cvalid, const T* v) { if (cvalid > 0) p[0] = v[0]; }
};
template <typename T, int VEC>
using ChunkOf = typename std::conditional<VEC == 1, Chunk1<T>, Chunk<T, VEC>>::type;

// Position of key in the sorted a[lo, hi), or -1.
__device__ __forceinline__ int find_sorted(const uint32_t* a, int lo, int hi, uint32_t key) {
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

// Diagonal <w|H|w> in fp64 (Eq. (1)): eps_i (n_up + n_dn) + U_i n_up n_dn.
__device__ __forceinline__ double diag_f64(const HamParams& hp, uint32_t up, uint32_t dn) {
  if (hp.uniform) return hp.dtab[__popc(up & dn)];
  double d = 0.0;
  for (int i = 0; i < hp.n_sites; ++i) {
    const int u = (up >> i) & 1, v = (dn >> i) & 1;
    d += hp.eps[i] * double(u + v) + hp.U[i] * double(u & v);
  }
  return d;
}

template <typename T>
struct Acc;
// fp32 vectors: coefficient = hi + lo (two floats), two accumulators.
template <>
struct Acc<float> {
  float h, l;
  __device__ __forceinline__ void zero() { h = 0.f; l = 0.f; }
  __device__ __forceinline__ void fma(float ch, float cl, float x) {
    h = fmaf(ch, x, h);
    l = fmaf(cl, x, l);
  }
  __device__ __forceinline__ float value() const { return h + l; }
};
template <>
struct Acc<double> {
  double h;
  __device__ __forceinline__ void zero() { h = 0.0; }
  __device__ __forceinline__ void fma(double c, double, double x) { h = ::fma(c, x, h); }
  __device__ __forceinline__ double value() const { return h; }
};

template <typename T>
struct Coef {
  T hi, lo;
};

// Double-float accumulation in fp32 arithmetic: (h, l) += (chi + clo) v, the
// product split exactly by an FMA and added by Knuth's two-sum followed by a
// fast renormalisation (Dekker), so (h + l) carries about 46 significant bits.
// Every operation is an explicitly rounded intrinsic: no contraction, the same
// bits wherever the step runs.  fp32 Ritz vectors are summed this way (GB300
// runs fp64 arithmetic and fp32 -> fp64 conversions at a small fraction of the
// fp32 rate, which made an fp64 sum of fp32 Krylov vectors ALU-bound).
__device__ __forceinline__ void df_fma(float& h, float& l, float chi, float clo, float v) {
  const float ph = __fmul_rn(chi, v);
  float pl = __fmaf_rn(chi, v, -ph);
  pl = __fmaf_rn(clo, v, pl);
  const float s = __fadd_rn(h, ph);
  const float bb = __fsub_rn(s, h);
  float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
  e = __fadd_rn(e, __fadd_rn(l, pl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// (h, l) += x in double-float (two-sum, then the fast renormalisation)
__device__ __forceinline__ void df_add(float& h, float& l, float x) {
  const float s = __fadd_rn(h, x);
  const float bb = __fsub_rn(s, h);
  float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  e = __fadd_rn(e, l);
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// fp64 coefficient c as (hi, lo) floats: hi = fl32(c), lo = fl32(c - hi)
__host__ __device__ __forceinline__ float2 split_coef(double c) {
  const float hi = float(c);
  return make_float2(hi, float(c - double(hi)));
}

template <typename T>
__device__ __forceinline__ Coef<T> bond_coef(const float* thi, const float* tlo, const double* t64, int b,
                                             int sign);
template <>
__device__ __forceinline__ Coef<float> bond_coef<float>(const float* thi, const float* tlo, const double*, int b,
                                                        int sign) {
  return Coef<float>{sign ? -thi[b] : thi[b], sign ? -tlo[b] : tlo[b]};
}
template <>
__device__ __forceinline__ Coef<double> bond_coef<double>(const float*, const float*, const double* t64, int b,
                                                          int sign) {
  return Coef<double>{sign ? -t64[b] : t64[b], 0.0};
}

template <typename T>
__device__ __forceinline__ Coef<T> diag_coef(const HamParams& hp, uint32_t up, uint32_t dn);
template <>
__device__ __forceinline__ Coef<float> diag_coef<float>(const HamParams& hp, uint32_t up, uint32_t dn) {
  if (hp.uniform) {
    const int k = __popc(up & dn);
    return Coef<float>{hp.dtab_hi[k], hp.dtab_lo[k]};
  }
  const double d = diag_f64(hp, up, dn);
  const float h = float(d);
  return Coef<float>{h, float(d - double(h))};
}
template <>
__device__ __forceinline__ Coef<double> diag_coef<double>(const HamParams& hp, uint32_t up, uint32_t dn) {
  return Coef<double>{diag_f64(hp, up, dn), 0.0};
}

}  // namespace
}  // namespace mcd
