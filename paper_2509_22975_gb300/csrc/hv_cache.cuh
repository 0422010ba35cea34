// Definitions shared by the connection-cache kernels (hv_cache.cu: record
// build and one-column streaming H~v; hv_cache_cols.cu: many columns):
// record formats, kernel arguments and the per-state record sum.
#pragma once

#include "hv_common.cuh"

namespace mcd {
namespace {

constexpr int kCT = 256;                     // threads of the build and multi-column kernels
constexpr int kCWarps = kCT / 32;
constexpr int kCItem = 512;                  // states per work item (at most, unless one block is larger)
constexpr int kLaneBytes = 8;                // bytes of a lane's records in one group
constexpr int kGroup = 32 * kLaneBytes;      // bytes of one record group (256)
constexpr int kSliceMap = 64;                // bytes of a slice's lane map (32 x u16)
constexpr uint16_t kNoState = 0xFFFFu;
constexpr int kBuildStageWords = 12288;      // minor words staged by the build kernels (48 KiB)
constexpr int kMStageBytes = 48 * 1024;      // staged x rows of the multi-column kernel
constexpr int kMaxCount = 512;               // records of one state in one pass (n_bonds <= 496)
constexpr uint32_t kSpinLimit = 1u << 22;    // polls of an mbarrier before a wait gives up
constexpr uint32_t kTestSpinLimit = 1u << 12;  // the same in a time-out test (MCD_OPT_WAIT_TEST)

template <typename R>
struct Rec;
template <>
struct Rec<uint16_t> {
  static constexpr int kPer = kLaneBytes / 2;   // records per lane per group
  static constexpr uint32_t kSent = 0xFFFFu;     // padding
  static constexpr uint32_t kMaxStage = 0x3FFFu; // positions 0 .. 0x3FFE (0x3FFF + sign + class 1 = padding)
  static constexpr int kMaxCls = 2;
  __host__ __device__ static uint32_t make(uint32_t q, uint32_t neg, uint32_t cls) {
    return q | (neg << 14) | (cls << 15);
  }
  __device__ static uint32_t pos(uint32_t r) { return r & 0x3FFFu; }
  __device__ static bool neg(uint32_t r) { return (r >> 14) & 1u; }
  __device__ static uint32_t cls(uint32_t r) { return r >> 15; }
};
template <>
struct Rec<uint32_t> {
  static constexpr int kPer = kLaneBytes / 4;
  static constexpr uint32_t kSent = 0xFFFFFFFFu;
  static constexpr uint32_t kMaxStage = 0x3FFFFFu;
  static constexpr int kMaxCls = 512;
  __host__ __device__ static uint32_t make(uint32_t q, uint32_t neg, uint32_t cls) {
    return q | (neg << 22) | (cls << 23);
  }
  __device__ static uint32_t pos(uint32_t r) { return r & 0x3FFFFFu; }
  __device__ static bool neg(uint32_t r) { return (r >> 22) & 1u; }
  __device__ static uint32_t cls(uint32_t r) { return r >> 23; }
};

struct CArgs {
  const void* x;
  void* y;
  const void* xb;                // pass B of the streaming kernel: x in layout order
  int x_layout;                  // many-column kernel: rows of x are in this layout's order
  void* yb;                      // streaming kernels: pass B's part of y (basis order), read by pass A
  int ncols, ld;
  int ncp;                       // staged row stride (elements)
  int xs_cap;                    // staged elements (multi-column) / minor words (build)
  int off_xs;                    // byte offset of the staging area in dynamic shared memory
  int n_sites;
  int64_t n;                     // states
  int64_t x_bytes;               // bytes of x the streaming kernel may read from its base
  const uint64_t* words;         // basis words (diagonal of pass A)
  const uint32_t* minor;
  const uint32_t* blk_off;
  const uint32_t* perm;          // pass B: layout position -> basis index
  const CItem* items;
  int64_t n_items;
  const uint32_t* col;           // [n_slices + 1] first record group of each slice
  const uint16_t* smap;          // [n_slices * 32] lane -> state of the item
  void* rec;
  const double* c64;             // [n_cls]
  const float* chi;
  const float* clo;
  int n_cls;
  double* dot_partials;
  unsigned int* ticket;
  double* dot_out;
  unsigned int* err;
  const uint4* units;            // many-column kernel: {first item, sb, stage rows, col0 | G | flags | items}
  int64_t n_units;
  uint32_t spin_limit;           // polls of an mbarrier before a wait gives up
  int64_t withhold;              // time-out test: item whose copies are not issued (-1 none)
  unsigned int* sched;           // streaming kernel: [0] next work item to claim, [1] CTAs done (both 0 between launches)
  // build
  const uint16_t* bond_cls;      // [n_bonds] record class of each bond
  uint16_t* cnt;                 // [n] records of each state
  uint32_t* wid;                 // [n_slices] groups of each slice
  uint16_t* smap_out;
  unsigned long long* nconn;     // found hops
};

// ---- apply --------------------------------------------------------------------------

// Slice of a work item for the consumer warp at position wpos of nw, on its
// pass `pass` over the item: an item's slices are sorted longest first, and
// the passes run forwards and backwards in turn (serpentine), so the warps
// that take a further slice are those whose previous one was shortest.
__device__ __forceinline__ int serp_slice(int pass, int wpos, int nw) {
  return pass * nw + ((pass & 1) ? nw - 1 - wpos : wpos);
}

__device__ __forceinline__ float flip_sign(float x, uint32_t sg) { return __int_as_float(__float_as_int(x) ^ int(sg)); }
__device__ __forceinline__ double flip_sign(double x, uint32_t sg) {
  return __longlong_as_double(__double_as_longlong(x) ^ (static_cast<long long>(sg) << 32));
}

template <typename T>
__device__ __forceinline__ T coef_hi(const double* c64, const float* chi, int c) {
  return sizeof(T) == 4 ? T(chi[c]) : T(c64[c]);
}
template <typename T>
__device__ __forceinline__ T coef_lo(const float* clo, int c) {
  return sizeof(T) == 4 ? T(clo[c]) : T(0);
}

// acc += sum over the records of one state of t_class sign x[target] (VEC
// columns).  rp = the lane's 8 bytes in the state's first group (shared or
// global memory); ng groups, 256 bytes apart.  gather(q, v) loads the VEC
// values of stage row q.  kU groups are loaded before any is used.
template <typename T, typename R, int VEC, int kU, typename Gather>
__device__ __forceinline__ void state_sum(const unsigned char* rp, int ng, int n_cls, const double* c64,
                                          const float* chi, const float* clo, Gather gather, Acc<T> (&acc)[VEC]) {
  using RR = Rec<R>;
  T s0[VEC], s1[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) s0[u] = s1[u] = T(0);
  int cur = -1;   // class of the running sum (4-byte records)
  for (int gb = 0; gb < ng; gb += kU, rp += kU * kGroup) {
    uint2 pks[kU];
#pragma unroll
    for (int v = 0; v < kU; ++v)
      pks[v] = gb + v < ng ? *reinterpret_cast<const uint2*>(rp + v * kGroup) : make_uint2(~0u, ~0u);
#pragma unroll
    for (int v = 0; v < kU; ++v) {
      const uint2 pk = pks[v];
      uint32_t r[RR::kPer];
      if constexpr (sizeof(R) == 2) {
        r[0] = pk.x & 0xFFFFu;
        r[1] = pk.x >> 16;
        r[2] = pk.y & 0xFFFFu;
        r[3] = pk.y >> 16;
      } else {
        r[0] = pk.x;
        r[1] = pk.y;
      }
      if (r[0] == RR::kSent) continue;   // padding is trailing: the rest of the group is padding
      T xv[RR::kPer][VEC];
#pragma unroll
      for (int h = 0; h < RR::kPer; ++h) {
        if (r[h] != RR::kSent) {
          gather(int(RR::pos(r[h])), xv[h]);
        } else {
#pragma unroll
          for (int u = 0; u < VEC; ++u) xv[h][u] = T(0);
        }
      }
#pragma unroll
      for (int h = 0; h < RR::kPer; ++h) {
        if constexpr (sizeof(R) == 2) {
          // branch-free: the sign flips the sign bit of x (exact); every hop
          // goes into s0, class-1 hops also into s1 (class 0 = s0 - s1 at
          // the end); padding adds a zero (exact)
          const bool c1 = (r[h] >> 15) & 1u;
          const uint32_t sg = (r[h] << 17) & 0x80000000u;
#pragma unroll
          for (int u = 0; u < VEC; ++u) {
            const T v = flip_sign(xv[h][u], sg);
            s0[u] += v;
            s1[u] += c1 ? v : T(0);
          }
        } else {
          if (r[h] == RR::kSent) continue;
          const bool ng_ = RR::neg(r[h]);
          const int cl = int(RR::cls(r[h]));
          if (cl != cur) {
            if (cur >= 0) {
              const T ch = coef_hi<T>(c64, chi, cur), cl_ = coef_lo<T>(clo, cur);
#pragma unroll
              for (int u = 0; u < VEC; ++u) {
                acc[u].fma(ch, cl_, s0[u]);
                s0[u] = T(0);
              }
            }
            cur = cl;
          }
#pragma unroll
          for (int u = 0; u < VEC; ++u) s0[u] += ng_ ? -xv[h][u] : xv[h][u];
        }
      }
    }
  }
  if constexpr (sizeof(R) == 2) {
    if (n_cls > 0) {
      const T ch = coef_hi<T>(c64, chi, 0), cl_ = coef_lo<T>(clo, 0);
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[u].fma(ch, cl_, s0[u] - s1[u]);
    }
    if (n_cls > 1) {
      const T ch = coef_hi<T>(c64, chi, 1), cl_ = coef_lo<T>(clo, 1);
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[u].fma(ch, cl_, s1[u]);
    }
  } else if (cur >= 0) {
    const T ch = coef_hi<T>(c64, chi, cur), cl_ = coef_lo<T>(clo, cur);
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc[u].fma(ch, cl_, s0[u]);
  }
}

template <typename T>
__device__ __forceinline__ Coef<T> diag_of(const HamParams& hp, const float* dhi, const float* dlo,
                                           const double* d64, uint32_t up, uint32_t dn) {
  if (hp.uniform) {
    const int nu = __popc(up & dn);
    return Coef<T>{sizeof(T) == 4 ? T(dhi[nu]) : T(d64[nu]), sizeof(T) == 4 ? T(dlo[nu]) : T(0)};
  }
  return diag_coef<T>(hp, up, dn);
}

// ---- mbarrier and bulk copy (PTX) -----------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// waits for the phase of the given parity; false when `limit` polls were not enough
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// 16-byte asynchronous copy global -> shared (both 16-byte aligned), L2 only
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// one arrival on bar once every cp.async this thread issued so far has landed
// (counts toward the barrier's expected arrivals)
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ---- host ------------------------------------------------------------------------

// (re)allocates p to at least need bytes, stream-ordered
inline cudaError_t grow_bytes(void*& p, int64_t& cap, int64_t need, cudaStream_t s) {
  if (p && cap >= need) return cudaSuccess;
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMallocAsync(&p, size_t(std::max<int64_t>(need, 16)), s);
  if (e != cudaSuccess) {
    p = nullptr;
    return e;
  }
  cap = need;
  return cudaSuccess;
}

inline void fill_args(mcd_ctx* c, const Layout& L, CArgs& a) {
  const ConnCache& cc = L.cc;
  a = CArgs{};
  a.n_sites = c->n;
  a.n = L.n;
  a.words = c->idx.words;
  a.minor = L.minor;
  a.blk_off = L.blk_off;
  a.perm = L.perm;
  a.items = cc.items;
  a.n_items = cc.n_items;
  a.col = cc.col;
  a.smap = cc.smap;
  a.rec = cc.rec;
  a.c64 = cc.c64;
  a.chi = cc.chi;
  a.clo = cc.clo;
  a.n_cls = cc.n_cls;
  a.err = cc.err;
  a.spin_limit = kSpinLimit;
  a.withhold = -1;
}

inline int cls_bytes(mcd_ctx* c) {
  int off = 0;
  for (Layout* L : {&c->idx.B, &c->idx.A}) off = std::max(off, L->cc.n_cls * 16);
  return (off + 127) & ~127;
}

}  // namespace
}  // namespace mcd
