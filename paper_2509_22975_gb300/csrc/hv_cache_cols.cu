// Connection-cache H~V for many columns (the blocked products of band
// Lanczos, App. C) and for one column with a row stride.
//
// Many columns: a persistent, warp-specialised kernel per pass.  Its work
// units are (work item, column tile) pairs: the tile width of an item is the
// widest, up to 8 chunks of 16 bytes, whose x rows of the item's stage range
// (the blocks its hop targets lie in) fit one stage of shared memory, so the
// large blocks are staged too, a few columns at a time.  Four producer warps
// fill each stage: one thread moves the item's records, lane map, slice
// offsets and per-state words (pass A) or basis indices (pass B) with bulk
// asynchronous copies, and all 128 gather the x rows of the tile with 16-byte
// cp.async copies, straight from the caller's X (pass B through the
// permutation, so X is never copied into the dn-major order); the stage's
// mbarrier completes when the bytes and every copy have landed.  Twelve
// consumer warps then read shared memory only: G lanes share a state, each
// owning one 16-byte chunk of the tile, and sum the state's records per
// amplitude class without branches (sign and class as multipliers of +-1 or
// 0, padding records pointed at a zero row).  Pass B writes its part of each
// row of Y through the permutation; pass A adds its part and the diagonal.
// Items whose stage rows do not fit even one chunk wide gather from global
// memory (the block is then read from L2).
//
// One column with a row stride (or misaligned columns): a CTA per item
// stages the x rows of the item's stage range when they fit and gathers
// through the permutation in pass B.  The records and their layout are those
// of hv_cache.cu.
#include <atomic>
#include <algorithm>
#include <cstring>
#include <vector>

#include "hv_cache.cuh"

namespace mcd {
namespace {

// ---- many columns: pipelined tiles ------------------------------------------

// Work unit: the items of one stage range (a run of whole blocks, or every
// piece of one large block) and a tile of the columns.  units[u] = {first
// item, sb, stage rows, col0 | G << 16 | x in global memory << 20 | items << 21}:
// the tile is columns [col0, col0 + G * VEC) (VEC = 16 bytes of elements), G
// lanes per state.  x rows of a unit are staged once for all its items.
constexpr int kTCons = 12;                      // consumer warps
constexpr int kTXProd = 3;                      // warps that stage x tiles
constexpr int kTThreads = 32 * (kTCons + 1 + kTXProd);   // + one warp whose lane 0 moves the records
constexpr int kTRecBytes = 20 * 1024;           // records of one item per record stage
constexpr int kTMapBytes = (kCItem / 32) * kSliceMap;
constexpr int kTColBytes = 128;                 // slice offsets (17 + alignment)
constexpr int kTAuxBytes = kCItem * 8 + 16;     // basis word (pass A) or basis index (pass B) per state
constexpr int kTOffMap = kTRecBytes;
constexpr int kTOffCol = kTOffMap + kTMapBytes;
constexpr int kTOffAux = kTOffCol + kTColBytes;
constexpr int kTRStageBytes = kTOffAux + kTAuxBytes;
constexpr int kTXBytes = 60 * 1024;             // x tile: stage rows + one zero row
constexpr int kTStages = 2;                     // record stages (one x buffer: two CTAs per SM overlap)
constexpr int kTSmem = kTStages * kTRStageBytes + kTXBytes;
static_assert(kTOffCol % 16 == 0 && kTOffAux % 16 == 0 && kTRStageBytes % 16 == 0 && kTXBytes % 16 == 0,
              "stage buffers on 16-byte boundaries");
constexpr int kTMaxG = 8;                       // chunks (lanes) per state
constexpr int kTMaxItems = 2047;                // items of one unit

// pass B gathering from global memory: the stage range's permutation
// entries (plus alignment) fit the x buffer
__host__ __device__ __forceinline__ bool perm_fits(int nst) { return int64_t(nst) * 4 + 32 <= kTXBytes; }

struct TRMeta {
  CItem it;
  uint32_t rdirect;   // the records are read from global memory
  int coff, aoff;     // first slice offset / state entry inside the staged spans
};

__device__ __forceinline__ uint32_t unit_col0(const uint4& u) { return u.w & 0xFFFFu; }
__device__ __forceinline__ int unit_g(const uint4& u) { return int((u.w >> 16) & 0xFu); }
__device__ __forceinline__ bool unit_xdirect(const uint4& u) { return ((u.w >> 20) & 1u) != 0u; }
__device__ __forceinline__ uint32_t unit_items(const uint4& u) { return u.w >> 21; }

// acc += sum over the 2-byte records of one state of t_class sign x[target]
// (VEC columns).  rp = the lane's 8 bytes in the state's first group; ng
// groups, 256 bytes apart; gather(q, v) loads the VEC values of stage row q,
// and row `zrow` (<= the largest position) is zero: padding records point
// there.  Every record goes into s0 with its sign, class-1 records also into
// s1 (class 0 = s0 - s1): the sign and class are multipliers of +-1 and 0, so
// the sums are those of sign flips and selections, exactly.
template <typename T>
__device__ __forceinline__ T unit_sign(uint32_t r);   // +-1 from bit 14 of a record
template <>
__device__ __forceinline__ float unit_sign<float>(uint32_t r) {
  return __int_as_float(int(0x3F800000u | ((r & 0x4000u) << 17)));
}
template <>
__device__ __forceinline__ double unit_sign<double>(uint32_t r) {
  return __longlong_as_double(static_cast<long long>(0x3FF0000000000000ull | (uint64_t(r & 0x4000u) << 49)));
}
template <typename T>
__device__ __forceinline__ T keep_if_class1(T sg, uint32_t r);   // sg for class 1 (bit 15), else 0
template <>
__device__ __forceinline__ float keep_if_class1<float>(float sg, uint32_t r) {
  return __int_as_float(__float_as_int(sg) & (int(r << 16) >> 31));
}
template <>
__device__ __forceinline__ double keep_if_class1<double>(double sg, uint32_t r) {
  return __longlong_as_double(__double_as_longlong(sg) & static_cast<long long>(int(r << 16) >> 31));
}

template <typename T, int VEC, typename Gather>
__device__ __forceinline__ void state_sum16(const unsigned char* rp, int ng, uint32_t zrow, int n_cls,
                                            const double* c64, const float* chi, const float* clo, Gather gather,
                                            Acc<T> (&acc)[VEC]) {
  T s0[VEC], s1[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) s0[u] = s1[u] = T(0);
  uint2 pk = ng > 0 ? *reinterpret_cast<const uint2*>(rp) : make_uint2(~0u, ~0u);
  for (int gb = 0; gb < ng; ++gb) {
    const uint2 cur = pk;
    rp += kGroup;
    if (gb + 1 < ng) pk = *reinterpret_cast<const uint2*>(rp);   // next group in flight
    if ((cur.x & 0xFFFFu) == 0xFFFFu) break;   // padding is trailing: the rest of the state is padding
    const uint32_t r[4] = {cur.x & 0xFFFFu, cur.x >> 16, cur.y & 0xFFFFu, cur.y >> 16};
    T xv[4][VEC];
#pragma unroll
    for (int h = 0; h < 4; ++h) gather(int(min(r[h] & 0x3FFFu, zrow)), xv[h]);   // padding: 0x3FFF -> zero row
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const T sg = unit_sign<T>(r[h]);
      const T sg1 = keep_if_class1<T>(sg, r[h]);
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        s0[u] = fma(sg, xv[h][u], s0[u]);
        s1[u] = fma(sg1, xv[h][u], s1[u]);
      }
    }
  }
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
}

template <typename T>
__device__ __forceinline__ void load16(const T* p, T* v) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  memcpy(v, &u, 16);
}

// One pass of Y = H~ X over the work units blockIdx.x + i gridDim.x (largest
// first).  Three roles: kTXProd warps stage the x tile of unit i into x buffer
// i % 2 (cp.async, completion on xfull); lane 0 of the record warp moves each
// item's records, lane map, slice offsets and per-state words or indices into
// record stage (item count) % 2 with bulk copies (rfull); the kTCons consumer
// warps take unit i's items one by one from shared memory only, releasing
// each record stage (rempty) and, after the last item, the x buffer (xempty).
// Every wait is bounded; a wait that gives up ends the CTA's work and sets the
// error word after its copies have landed.
template <typename T, bool PASS_A>
__global__ void __launch_bounds__(kTThreads, 2) hv_tile_kernel(const CArgs a, const HamParams hp) {
  constexpr int VEC = 16 / int(sizeof(T));
  using C = ChunkOf<T, VEC>;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ __align__(8) uint64_t s_xfull, s_xempty, s_rfull[kTStages], s_rempty[kTStages];
  __shared__ uint4 s_unit;
  __shared__ TRMeta s_rmeta[kTStages];
  __shared__ float s_dhi[kMaxSites + 1], s_dlo[kMaxSites + 1];
  __shared__ double s_d64[kMaxSites + 1];
  unsigned char* s_rst = s_dyn;                                  // record stages
  unsigned char* s_xbuf = s_dyn + kTStages * kTRStageBytes;      // x buffer
  double* s_c64 = reinterpret_cast<double*>(s_dyn + kTSmem);
  float* s_chi = reinterpret_cast<float*>(s_c64 + a.n_cls);
  float* s_clo = s_chi + a.n_cls;
  for (int i = threadIdx.x; i < a.n_cls; i += kTThreads) {
    s_c64[i] = a.c64[i];
    s_chi[i] = a.chi[i];
    s_clo[i] = a.clo[i];
  }
  if (threadIdx.x <= kMaxSites) {
    s_dhi[threadIdx.x] = hp.dtab_hi[threadIdx.x];
    s_dlo[threadIdx.x] = hp.dtab_lo[threadIdx.x];
    s_d64[threadIdx.x] = hp.dtab[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    mbar_init(&s_xfull, 32 * kTXProd + 1);
    mbar_init(&s_xempty, kTCons);
    for (int s = 0; s < kTStages; ++s) {
      mbar_init(&s_rfull[s], 1);
      mbar_init(&s_rempty[s], kTCons);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n_my = blockIdx.x < a.n_units ? (a.n_units - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  auto unit_at = [&](int64_t i) { return a.units[blockIdx.x + i * int64_t(gridDim.x)]; };
  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const unsigned char* recg = static_cast<const unsigned char*>(a.rec);
  const int64_t ld = a.ld;
  bool failed = false;
  int64_t issued[kTStages];   // record thread: last item count whose bulk copies went into each stage
  for (int s = 0; s < kTStages; ++s) issued[s] = -1;

  if (warp > kTCons) {
    // x tiles: the x buffer holds unit i once the consumers are done with unit i - 1
    const int xt = (warp - kTCons - 1) * 32 + lane;
    uint4 nxt = n_my > 0 ? unit_at(0) : make_uint4(0, 0, 0, 0);
    for (int64_t i = 0; i < n_my; ++i) {
      const uint4 u = nxt;
      if (i + 1 < n_my) nxt = unit_at(i + 1);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&s_xempty, uint32_t(i & 1) ^ 1u, a.spin_limit) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        failed = true;
        break;
      }
      const uint32_t sb = u.y, col0 = unit_col0(u);
      const int nst = int(u.z), G = unit_g(u), tw = G * VEC;
      const bool xdirect = unit_xdirect(u);
      T* xs = reinterpret_cast<T*>(s_xbuf);
      if (!xdirect) {
        // rows of the stage range, columns [col0, col0 + tw): G consecutive
        // threads copy one row (its 16-byte chunks side by side); pass B's rows
        // through the permutation, kPF of them loaded before any copy
        constexpr int kPF = 4;
        constexpr int kXT = 32 * kTXProd;
        const int rpp = kXT / G;                 // rows per round
        const int tr = xt / G, tc = xt - tr * G;
        if (tr < rpp) {
          for (int q0 = tr; q0 < nst; q0 += kPF * rpp) {
            int64_t rows[kPF];
#pragma unroll
            for (int v = 0; v < kPF; ++v) {
              const int q = q0 + v * rpp;
              rows[v] = PASS_A ? int64_t(sb) + q : (q < nst ? int64_t(__ldg(a.perm + sb + q)) : 0);
            }
#pragma unroll
            for (int v = 0; v < kPF; ++v) {
              const int q = q0 + v * rpp;
              if (q < nst) cp_async16(xs + q * tw + tc * VEC, x + rows[v] * ld + col0 + tc * VEC);
            }
          }
        }
      }
      cp_async_mbar_arrive(&s_xfull);
      const int64_t unit = blockIdx.x + i * int64_t(gridDim.x);
      if (xt == 0 && unit != a.withhold) {   // time-out test: no arrival for the withheld unit
        s_unit = u;
        if (!xdirect) {
          for (int j = 0; j < G; ++j) *reinterpret_cast<uint4*>(xs + nst * tw + j * VEC) = make_uint4(0, 0, 0, 0);
          mbar_arrive(&s_xfull);
        } else if (!PASS_A && perm_fits(nst)) {
          // rows gathered from global memory: the stage range's basis indices
          // in the x buffer instead (one bulk copy of whole 16-byte units)
          const int64_t plo = (int64_t(sb) * 4) & ~int64_t(15);
          const int64_t phi = ((int64_t(sb) + nst) * 4 + 15) & ~int64_t(15);
          mbar_arrive_tx(&s_xfull, uint32_t(phi - plo));
          bulk_g2s(s_xbuf, reinterpret_cast<const unsigned char*>(a.perm) + plo, uint32_t(phi - plo), &s_xfull);
        } else {
          mbar_arrive(&s_xfull);
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's copies land before the CTA exits
  } else if (warp == kTCons) {
    // records of every item of every unit, in order
    if (lane == 0 && n_my > 0) {
      int64_t i = 0, ri = 0;
      uint32_t j = 0;
      uint4 u = unit_at(0);
      CItem it = a.items[u.x];
      while (i < n_my) {
        // the next (unit, item) descriptors, loaded while this item is issued
        int64_t i2 = i;
        uint32_t j2 = j + 1;
        uint4 u2 = u;
        if (j2 >= unit_items(u)) {
          i2 = i + 1;
          j2 = 0;
          if (i2 < n_my) u2 = unit_at(i2);
        }
        CItem it2 = it;
        if (i2 < n_my) it2 = a.items[u2.x + j2];
        const int rs = int(ri & 1);
        if (!mbar_wait(&s_rempty[rs], uint32_t((ri >> 1) & 1) ^ 1u, a.spin_limit)) {
          failed = true;
          break;
        }
        unsigned char* stage = s_rst + rs * kTRStageBytes;
        const int nsl = int((it.hi - it.lo + 31) / 32);
        const uint32_t rb = (it.g1 - it.g0) * uint32_t(kGroup);
        const bool rdirect = rb > uint32_t(kTRecBytes);
        const uint32_t mb = uint32_t(nsl) * kSliceMap;
        constexpr int64_t es_aux = PASS_A ? 8 : 4;
        const int64_t clo = (int64_t(it.slice0) * 4) & ~int64_t(15);
        const int64_t chi = ((int64_t(it.slice0) + nsl + 1) * 4 + 15) & ~int64_t(15);
        const int64_t alo = (int64_t(it.lo) * es_aux) & ~int64_t(15);
        const int64_t ahi = (int64_t(it.hi) * es_aux + 15) & ~int64_t(15);
        TRMeta m;
        m.it = it;
        m.rdirect = rdirect ? 1u : 0u;
        m.coff = int((int64_t(it.slice0) * 4 - clo) / 4);
        m.aoff = int((int64_t(it.lo) * es_aux - alo) / es_aux);
        s_rmeta[rs] = m;
        const uint32_t bytes = (rdirect ? 0u : rb) + mb + uint32_t(chi - clo) + uint32_t(ahi - alo);
        mbar_arrive_tx(&s_rfull[rs], bytes);
        if (!rdirect && rb) bulk_g2s(stage, recg + int64_t(it.g0) * kGroup, rb, &s_rfull[rs]);
        bulk_g2s(stage + kTOffMap, a.smap + int64_t(it.slice0) * 32, mb, &s_rfull[rs]);
        bulk_g2s(stage + kTOffCol, reinterpret_cast<const unsigned char*>(a.col) + clo, uint32_t(chi - clo),
                 &s_rfull[rs]);
        const unsigned char* aux =
            PASS_A ? reinterpret_cast<const unsigned char*>(a.words) : reinterpret_cast<const unsigned char*>(a.perm);
        bulk_g2s(stage + kTOffAux, aux + alo, uint32_t(ahi - alo), &s_rfull[rs]);
        issued[rs] = ri;
        ++ri;
        i = i2;
        j = j2;
        u = u2;
        it = it2;
      }
    }
  } else {
    // consumers
    int64_t ri = 0;
    for (int64_t i = 0; i < n_my && !failed; ++i) {
      if (!mbar_wait(&s_xfull, uint32_t(i & 1), a.spin_limit)) {
        failed = true;
        break;
      }
      const uint4 u = s_unit;
      const uint32_t sb = u.y, col0 = unit_col0(u), nit = unit_items(u);
      const int nst = int(u.z), G = unit_g(u), tw = G * VEC;
      const bool xdirect = unit_xdirect(u);
      const int spw = 32 / G;                      // states of a slice taken at once by the warp
      const int tg = lane / G, g = lane - tg * G;
      const bool lane_ok = tg < spw;
      const int col = int(col0) + g * VEC;
      const int cvalid = a.ncols - col;
      const T* xs = reinterpret_cast<const T*>(s_xbuf) + g * VEC;
      // pass B with global gathers: the staged permutation entries (the span
      // starts on a 16-byte boundary, sb & 3 entries before perm[sb])
      const bool pstaged = !PASS_A && xdirect && perm_fits(nst);
      const uint32_t* sperm = reinterpret_cast<const uint32_t*>(s_xbuf) + (sb & 3u);
      auto gather = [&](int q, T* v) {
        if (!xdirect) {
          load16(xs + q * tw, v);
        } else if (q >= nst) {
#pragma unroll
          for (int w = 0; w < VEC; ++w) v[w] = T(0);
        } else {
          const int64_t row = PASS_A ? int64_t(sb) + q : int64_t(pstaged ? sperm[q] : __ldg(a.perm + sb + q));
          C::load(x + row * ld + col, cvalid, v);
        }
      };
      for (uint32_t j = 0; j < nit; ++j, ++ri) {
        const int rs = int(ri & 1);
        if (!mbar_wait(&s_rfull[rs], uint32_t((ri >> 1) & 1), a.spin_limit)) {
          failed = true;
          break;
        }
        const TRMeta& m = s_rmeta[rs];   // read in place: stable while the stage is held
        const CItem& it = m.it;
        const unsigned char* stage = s_rst + rs * kTRStageBytes;
        const uint32_t* colp = reinterpret_cast<const uint32_t*>(stage + kTOffCol) + m.coff;
        const uint16_t* mapp = reinterpret_cast<const uint16_t*>(stage + kTOffMap);
        const unsigned char* recb = m.rdirect ? recg + int64_t(it.g0) * kGroup : stage;
        const int nsl = int((it.hi - it.lo + 31) / 32);
        const bool wide = (it.flags & 1u) != 0u;
        // serpentine slice order, rotated from item to item (see serp_slice)
        const int wpos = (warp + kTCons - int((ri * 4) % kTCons)) % kTCons;
        for (int pass = 0;; ++pass) {
          const int sl = serp_slice(pass, wpos, kTCons);
          if (sl >= nsl) break;
          const uint32_t ga = colp[sl], gz = colp[sl + 1];
          const uint32_t locs = mapp[sl * 32 + lane];
          for (int t0 = 0; t0 < 32; t0 += spw) {
            const int t = t0 + tg;
            const uint16_t loc = uint16_t(__shfl_sync(0xffffffffu, locs, t & 31));
            if (!lane_ok || t >= 32 || loc == kNoState || cvalid <= 0) continue;
            const uint32_t k = it.lo + loc;
            T yk[VEC];
            if (PASS_A) C::load(y + int64_t(k) * ld + col, cvalid, yk);   // in flight during the record sum
            const unsigned char* rp = recb + int64_t(ga - it.g0) * kGroup + t * kLaneBytes;
            Acc<T> acc[VEC];
#pragma unroll
            for (int w = 0; w < VEC; ++w) acc[w].zero();
            if (wide)
              state_sum<T, uint32_t, VEC, 2>(rp, int(gz - ga), a.n_cls, s_c64, s_chi, s_clo, gather, acc);
            else
              state_sum16<T, VEC>(rp, int(gz - ga), uint32_t(nst), a.n_cls, s_c64, s_chi, s_clo, gather, acc);
            T out[VEC];
            if (PASS_A) {
              const uint64_t w = reinterpret_cast<const uint64_t*>(stage + kTOffAux)[m.aoff + loc];
              const uint32_t half = a.n_sites >= 32 ? 0xFFFFFFFFu : ((1u << a.n_sites) - 1u);
              const uint32_t up = uint32_t(w >> a.n_sites), dn = uint32_t(w) & half;
              T xk[VEC];
              gather(int(k - sb), xk);
              const Coef<T> dc = diag_of<T>(hp, s_dhi, s_dlo, s_d64, up, dn);
#pragma unroll
              for (int w2 = 0; w2 < VEC; ++w2) {
                acc[w2].fma(dc.hi, dc.lo, xk[w2]);
                out[w2] = acc[w2].value() + yk[w2];
              }
              C::store(y + int64_t(k) * ld + col, cvalid, out);
            } else {
              const uint32_t row = reinterpret_cast<const uint32_t*>(stage + kTOffAux)[m.aoff + loc];
#pragma unroll
              for (int w2 = 0; w2 < VEC; ++w2) out[w2] = acc[w2].value();
              C::store(y + int64_t(row) * ld + col, cvalid, out);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_rempty[rs]);
      }
      if (failed) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_xempty);
    }
  }
  const int any_failed = __syncthreads_or(failed ? 1 : 0);
  if (any_failed) {
    if (warp == kTCons && lane == 0) {
      // bulk copies still in flight land before the CTA's shared memory is released
      for (int s = 0; s < kTStages; ++s)
        if (issued[s] >= 0) mbar_wait(&s_rfull[s], uint32_t((issued[s] >> 1) & 1), a.spin_limit);
    }
    if (threadIdx.x == 0) atomicOr(a.err, 1u);
    __syncthreads();
  }
}

// Work units of a layout for rows of nch chunks of vec elements of es bytes:
// consecutive items of one stage range form a group; per group the widest
// tile (<= kTMaxG chunks, balanced over the row) whose stage rows plus the
// zero row fit an x buffer; groups that do not fit even one chunk wide gather
// from global memory, kTMaxG chunks at a time.  Largest groups first.
void make_units(const std::vector<uint2>& rng, int nch, int vec, int es, std::vector<uint4>& out) {
  struct U {
    uint4 u;
    uint64_t cost;
  };
  std::vector<U> tmp;
  const int gmax = std::min(kTMaxG, nch);
  size_t i = 0;
  while (i < rng.size()) {
    size_t j = i + 1;
    while (j < rng.size() && rng[j].x == rng[i].x && rng[j].y == rng[i].y && j - i < size_t(kTMaxItems)) ++j;
    const uint32_t sb = rng[i].x, nst = rng[i].y - rng[i].x;
    const int64_t r = int64_t(nst) + 1;
    int g = gmax;
    while (g > 1 && r * g * vec * es > kTXBytes) --g;
    const bool direct = r * g * vec * es > kTXBytes;
    if (direct) g = gmax;
    const int tiles = (nch + g - 1) / g;
    const int gb = (nch + tiles - 1) / tiles;
    for (int c0 = 0; c0 < nch; c0 += gb) {
      const int gg = std::min(gb, nch - c0);
      const uint32_t w = uint32_t(c0 * vec) | (uint32_t(gg) << 16) | (direct ? (1u << 20) : 0u) |
                         (uint32_t(j - i) << 21);
      tmp.push_back(U{make_uint4(uint32_t(i), sb, nst, w), uint64_t(nst) * uint64_t(gg)});
    }
    i = j;
  }
  std::stable_sort(tmp.begin(), tmp.end(), [](const U& p, const U& q) { return p.cost > q.cost; });
  out.resize(tmp.size());
  for (size_t k = 0; k < tmp.size(); ++k) out[k] = tmp[k].u;
}

template <typename T>
cudaError_t launch_tiles(mcd_ctx* c, const void* x, void* y, int ncols, int ld) {
  constexpr int VEC = 16 / int(sizeof(T));
  const int nch = (ncols + VEC - 1) / VEC;
  const int smem = kTSmem + cls_bytes(c);
  static std::atomic<int> configured{-1};   // per instantiation
  if (configured < smem) {
    cudaFuncSetAttribute(hv_tile_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(hv_tile_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    configured = smem;
  }
  const int key = nch * VEC * 16 + int(sizeof(T));
  for (int pass = 0; pass < 2; ++pass) {
    Layout& L = pass == 0 ? c->idx.B : c->idx.A;
    ConnCache& cc = L.cc;
    if (cc.units_key != key) {
      std::vector<uint4> u;
      make_units(c->stage_range[pass], nch, VEC, int(sizeof(T)), u);
      void* p = cc.units;
      int64_t cap = cc.units_cap * 16;
      cudaError_t e = grow_bytes(p, cap, int64_t(u.size()) * 16, c->stream);
      cc.units = static_cast<uint4*>(p);
      cc.units_cap = cap / 16;
      if (e == cudaSuccess && !u.empty())
        e = cudaMemcpyAsync(cc.units, u.data(), u.size() * 16, cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) {
        cc.units_key = -1;
        return e;
      }
      cc.n_units = int64_t(u.size());
      cc.units_key = key;
    }
    CArgs a;
    fill_args(c, L, a);
    a.x = x;
    a.y = y;
    a.ncols = ncols;
    a.ld = ld;
    a.units = cc.units;
    a.n_units = cc.n_units;
    if (c->wait_test_item >= 0) {
      a.spin_limit = kTestSpinLimit;
      if (pass == 1) a.withhold = c->wait_test_item;
    }
    if (a.n_units <= 0) continue;
    const int per_sm = smem <= 113 * 1024 ? 2 : 1;
    const int grid = int(std::min<int64_t>(a.n_units, int64_t(device_sms()) * per_sm));
    timing_begin(c, pass == 0 ? 0 : 1);
    if (pass == 0)
      hv_tile_kernel<T, false><<<grid, kTThreads, smem, c->stream>>>(a, *c->hp);
    else
      hv_tile_kernel<T, true><<<grid, kTThreads, smem, c->stream>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  c->wait_test_item = -1;   // the test option applies to one product
  return cudaSuccess;
}

// ---- one column with a row stride ------------------------------------------------

// CTA per item, x rows of the stage range staged with ordinary loads when they
// fit (pass B through the permutation), one lane per state.
template <typename T, bool PASS_A>
__global__ void __launch_bounds__(kCT) hv_cached_kernel(const CArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  double* s_c64 = reinterpret_cast<double*>(s_dyn);
  float* s_chi = reinterpret_cast<float*>(s_c64 + a.n_cls);
  float* s_clo = s_chi + a.n_cls;
  T* xs = reinterpret_cast<T*>(s_dyn + a.off_xs);
  __shared__ float s_dhi[kMaxSites + 1], s_dlo[kMaxSites + 1];
  __shared__ double s_d64[kMaxSites + 1];
  for (int i = threadIdx.x; i < a.n_cls; i += kCT) {
    s_c64[i] = a.c64[i];
    s_chi[i] = a.chi[i];
    s_clo[i] = a.clo[i];
  }
  if (threadIdx.x <= kMaxSites) {
    s_dhi[threadIdx.x] = hp.dtab_hi[threadIdx.x];
    s_dlo[threadIdx.x] = hp.dtab_lo[threadIdx.x];
    s_d64[threadIdx.x] = hp.dtab[threadIdx.x];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const unsigned char* recg = static_cast<const unsigned char*>(a.rec);
  const uint32_t half = a.n_sites >= 32 ? 0xFFFFFFFFu : ((1u << a.n_sites) - 1u);
  const int64_t ld = a.ld;

  for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const CItem it = a.items[item];
    const uint32_t sb = a.blk_off[it.b0], se = a.blk_off[it.b1 + 1];
    const int nst = int(se - sb);
    const bool staged = nst <= a.xs_cap;
    __syncthreads();   // the previous item's rows are no longer read
    if (staged) {
      for (int q = threadIdx.x; q < nst; q += kCT) {
        const int64_t row = PASS_A ? int64_t(sb) + q : int64_t(__ldg(a.perm + sb + q));
        xs[q] = x[row * ld];
      }
    }
    __syncthreads();
    const bool wide = (it.flags & 1u) != 0u;
    auto gather = [&](int q, T* v) {
      if (staged) {
        v[0] = xs[q];
      } else {
        const int64_t row = PASS_A ? int64_t(sb) + q : int64_t(__ldg(a.perm + sb + q));
        v[0] = x[row * ld];
      }
    };
    const int nsl = int((it.hi - it.lo + 31) / 32);
    for (int sl = warp; sl < nsl; sl += kCWarps) {
      const int64_t s = int64_t(it.slice0) + sl;
      const uint32_t ga = __ldg(a.col + s), gz = __ldg(a.col + s + 1);
      const uint16_t loc = __ldg(a.smap + s * 32 + lane);
      if (loc == kNoState) continue;                      // empty lanes are the slice's last ones
      const uint32_t k = it.lo + loc;
      const unsigned char* rp = recg + int64_t(ga) * kGroup + lane * kLaneBytes;
      Acc<T> acc[1];
      acc[0].zero();
      if (wide)
        state_sum<T, uint32_t, 1, 8>(rp, int(gz - ga), a.n_cls, s_c64, s_chi, s_clo, gather, acc);
      else
        state_sum<T, uint16_t, 1, 8>(rp, int(gz - ga), a.n_cls, s_c64, s_chi, s_clo, gather, acc);
      if (PASS_A) {
        const uint64_t w = __ldg(a.words + k);
        const uint32_t up = uint32_t(w >> a.n_sites), dn = uint32_t(w) & half;
        T xk;
        gather(int(k - sb), &xk);
        const Coef<T> dc = diag_of<T>(hp, s_dhi, s_dlo, s_d64, up, dn);
        acc[0].fma(dc.hi, dc.lo, xk);
        y[int64_t(k) * ld] = acc[0].value() + y[int64_t(k) * ld];
      } else {
        y[int64_t(__ldg(a.perm + k)) * ld] = acc[0].value();
      }
    }
  }
}

template <typename T>
cudaError_t launch_strided(mcd_ctx* c, const void* x, void* y, int ld) {
  const int off_xs = cls_bytes(c);
  const int smem = off_xs + kMStageBytes;
  static std::atomic<int> configured{-1};   // per instantiation
  if (configured < smem) {
    cudaFuncSetAttribute(hv_cached_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(hv_cached_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    configured = smem;
  }
  for (int pass = 0; pass < 2; ++pass) {
    const Layout& L = pass == 0 ? c->idx.B : c->idx.A;
    CArgs a;
    fill_args(c, L, a);
    a.x = x;
    a.y = y;
    a.ncols = 1;
    a.ld = ld;
    a.off_xs = off_xs;
    a.xs_cap = int(kMStageBytes / sizeof(T));
    if (a.n_items <= 0) continue;
    timing_begin(c, pass == 0 ? 0 : 1);
    if (pass == 0)
      hv_cached_kernel<T, false><<<int(a.n_items), kCT, smem, c->stream>>>(a, *c->hp);
    else
      hv_cached_kernel<T, true><<<int(a.n_items), kCT, smem, c->stream>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

namespace {

// the pipelined-tile kernel for these columns, or *used = false
cudaError_t apply_tiles(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, bool* used) {
  const bool f64 = dtype == MCD_F64;
  const int vec = f64 ? 2 : 4;
  const bool vec_ok = ld % vec == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(y) % 16 == 0 && (ncols + vec - 1) / vec * vec <= 65535;
  *used = vec_ok;
  if (!vec_ok) return cudaSuccess;
  return f64 ? launch_tiles<double>(c, x, y, ncols, ld) : launch_tiles<float>(c, x, y, ncols, ld);
}

// Time both many-column kernels on this product (each after its one-time
// preparation) and keep the faster for the column count and dtype; y holds
// the second kernel's (equally valid) result.
cudaError_t pick_and_apply(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, bool* used, int& pick) {
  cudaStream_t s = c->stream;
  for (auto& ev : c->tune_ev)
    if (!ev) {
      const cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return e;
    }
  cudaError_t e = cache_items_prepare(c, ncols, dtype);
  if (e != cudaSuccess) return e;
  // where more than a tenth of a pass's work items have stage ranges too long
  // for even one 16-byte column chunk in the x buffer, the tiles gather those
  // rows from L2 and lose to the CTA-per-item kernel (3x on the 6x4 basis):
  // no trial then
  for (int pass = 0; pass < 2; ++pass) {
    const std::vector<uint2>& rng = c->stage_range[pass];
    size_t direct = 0;
    for (const uint2& r : rng)
      if ((int64_t(r.y) - r.x + 1) * 16 > kTXBytes) ++direct;
    if (direct * 10 > rng.size()) {
      pick = 2;
      return cache_apply_items(c, x, y, ncols, ld, dtype, used);
    }
  }
  bool u1 = false, u2 = false;
  e = cudaEventRecord(c->tune_ev[0], s);
  if (e == cudaSuccess) e = apply_tiles(c, x, y, ncols, ld, dtype, &u1);   // also builds its work units
  if (e == cudaSuccess) e = cudaEventRecord(c->tune_ev[1], s);
  if (e == cudaSuccess) e = apply_tiles(c, x, y, ncols, ld, dtype, &u1);   // timed without the set-up
  if (e == cudaSuccess) e = cudaEventRecord(c->tune_ev[2], s);
  if (e != cudaSuccess) return e;
  float t_tiles = 0.f, t_items = 0.f;
  e = cudaEventSynchronize(c->tune_ev[2]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_tiles, c->tune_ev[1], c->tune_ev[2]);
  if (e == cudaSuccess) e = cudaEventRecord(c->tune_ev[0], s);
  if (e == cudaSuccess) e = cache_apply_items(c, x, y, ncols, ld, dtype, &u2);
  if (e == cudaSuccess) e = cudaEventRecord(c->tune_ev[1], s);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->tune_ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_items, c->tune_ev[0], c->tune_ev[1]);
  if (e != cudaSuccess) return e;
  if (!u2) {   // the item kernel does not take these columns: the tiles' result stands
    pick = 1;
    return apply_tiles(c, x, y, ncols, ld, dtype, used);
  }
  pick = t_tiles <= t_items ? 1 : 2;
  *used = true;
  return cudaSuccess;
}

}  // namespace

cudaError_t cache_apply_cols(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, bool* used) {
  *used = false;
  const bool f64 = dtype == MCD_F64;
  if (ncols == 1) {
    *used = true;
    return f64 ? launch_strided<double>(c, x, y, ld) : launch_strided<float>(c, x, y, ld);
  }
  if (c->hv_cols == 1 || ncols > 64) return apply_tiles(c, x, y, ncols, ld, dtype, used);
  if (c->hv_cols == 2) {
    cudaError_t e = cache_items_prepare(c, ncols, dtype);
    if (e != cudaSuccess) return e;
    return cache_apply_items(c, x, y, ncols, ld, dtype, used);
  }
  int& pick = c->cols_pick[ncols][f64 ? 1 : 0];
  if (pick == 1) return apply_tiles(c, x, y, ncols, ld, dtype, used);
  if (pick == 2) return cache_apply_items(c, x, y, ncols, ld, dtype, used);
  if (c->wait_test_item >= 0) return apply_tiles(c, x, y, ncols, ld, dtype, used);   // the test takes the tiles
  return pick_and_apply(c, x, y, ncols, ld, dtype, used, pick);
}

}  // namespace mcd
