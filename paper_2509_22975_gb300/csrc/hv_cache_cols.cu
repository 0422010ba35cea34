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
#include <algorithm>
#include <cstring>
#include <vector>

#include "hv_cache.cuh"

namespace mcd {
namespace {

// ---- many columns: pipelined tiles ------------------------------------------

constexpr int kTCons = 12;                      // consumer warps
constexpr int kTProd = 4;                       // producer warps
constexpr int kTThreads = 32 * (kTCons + kTProd);
constexpr int kTStages = 2;
constexpr int kTRecBytes = 24 * 1024;           // records of one item per stage
constexpr int kTMapBytes = (kCItem / 32) * kSliceMap;
constexpr int kTColBytes = 128;                 // slice offsets (17 + alignment)
constexpr int kTAuxBytes = kCItem * 8 + 16;     // basis word (pass A) or basis index (pass B) per state
constexpr int kTXBytes = 78 * 1024;             // x tile: stage rows + one zero row
constexpr int kTOffMap = kTRecBytes;
constexpr int kTOffCol = kTOffMap + kTMapBytes;
constexpr int kTOffAux = kTOffCol + kTColBytes;
constexpr int kTOffX = kTOffAux + kTAuxBytes;
constexpr int kTStageBytes = kTOffX + kTXBytes;
static_assert(kTOffCol % 16 == 0 && kTOffAux % 16 == 0 && kTOffX % 16 == 0 && kTStageBytes % 16 == 0,
              "stage buffers on 16-byte boundaries");
constexpr int kTMaxG = 8;                       // chunks (lanes) per state

struct TMeta {
  CItem it;
  uint32_t col0, G, flags;   // flags: 1 = records read from global memory, 2 = x rows too
  int coff, aoff;            // first slice offset / state entry inside the staged spans
};

// acc += sum over the 2-byte records of one state of t_class sign x[target]
// (VEC columns).  rp = the lane's 8 bytes in the state's first group; ng
// groups, 256 bytes apart; gather(q, v) loads the VEC values of stage row q,
// and row `zrow` is zero (padding records point there).  Every record goes
// into s0 with its sign, class-1 records also into s1 (class 0 = s0 - s1):
// the sign and class are multipliers of +-1 and 0, so the sums are those of
// sign flips and selections, exactly.
template <typename T, int VEC, int kU, typename Gather>
__device__ __forceinline__ void state_sum16(const unsigned char* rp, int ng, int zrow, int n_cls, const double* c64,
                                            const float* chi, const float* clo, Gather gather, Acc<T> (&acc)[VEC]) {
  T s0[VEC], s1[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) s0[u] = s1[u] = T(0);
  for (int gb = 0; gb < ng; gb += kU, rp += kU * kGroup) {
    uint2 pks[kU];
#pragma unroll
    for (int v = 0; v < kU; ++v)
      pks[v] = gb + v < ng ? *reinterpret_cast<const uint2*>(rp + v * kGroup) : make_uint2(~0u, ~0u);
#pragma unroll
    for (int v = 0; v < kU; ++v) {
      const uint2 pk = pks[v];
      if ((pk.x & 0xFFFFu) == 0xFFFFu) continue;   // padding is trailing: the rest of the group is padding
      const uint32_t r[4] = {pk.x & 0xFFFFu, pk.x >> 16, pk.y & 0xFFFFu, pk.y >> 16};
      T xv[4][VEC];
#pragma unroll
      for (int h = 0; h < 4; ++h) gather(r[h] == 0xFFFFu ? zrow : int(r[h] & 0x3FFFu), xv[h]);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const T sg = ((r[h] >> 14) & 1u) ? T(-1) : T(1);
        const T sg1 = ((r[h] >> 15) & 1u) ? sg : T(0);
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          s0[u] = fma(sg, xv[h][u], s0[u]);
          s1[u] = fma(sg1, xv[h][u], s1[u]);
        }
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

// One pass of Y = H~ X over the work units blockIdx.x + i gridDim.x.
// Stage i % kTStages holds unit i; full[st] completes when lane 0 of the
// first producer warp has announced the bulk bytes and every producer thread's
// cp.async copies have landed, empty[st] when the kTCons consumer warps are
// done with it.  Every wait is bounded; a wait that gives up sets the error
// word after this CTA's copies have landed.
template <typename T, bool PASS_A>
__global__ void __launch_bounds__(kTThreads, 1) hv_tile_kernel(const CArgs a, const HamParams hp) {
  constexpr int VEC = 16 / int(sizeof(T));
  using C = ChunkOf<T, VEC>;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ __align__(8) uint64_t s_full[kTStages], s_empty[kTStages];
  __shared__ TMeta s_meta[kTStages];
  __shared__ float s_dhi[kMaxSites + 1], s_dlo[kMaxSites + 1];
  __shared__ double s_d64[kMaxSites + 1];
  double* s_c64 = reinterpret_cast<double*>(s_dyn + kTStages * kTStageBytes);
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
    for (int s = 0; s < kTStages; ++s) {
      mbar_init(&s_full[s], 32 * kTProd + 1);
      mbar_init(&s_empty[s], kTCons);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n_my = blockIdx.x < a.n_units ? (a.n_units - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const unsigned char* recg = static_cast<const unsigned char*>(a.rec);
  const int64_t ld = a.ld;
  bool failed = false;
  int64_t issued[kTStages];   // first producer thread: last unit whose bulk copies went into each stage
  for (int s = 0; s < kTStages; ++s) issued[s] = -1;

  if (warp >= kTCons) {
    // producers
    const int pt = (warp - kTCons) * 32 + lane;
    for (int64_t i = 0; i < n_my; ++i) {
      const int st = int(i % kTStages);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&s_empty[st], uint32_t((i / kTStages) & 1) ^ 1u, a.spin_limit) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        failed = true;
        break;
      }
      const int64_t unit = blockIdx.x + i * int64_t(gridDim.x);
      const uint2 ud = a.units[unit];
      const CItem it = a.items[ud.x];
      const uint32_t col0 = ud.y & 0xFFFFu, G = (ud.y >> 16) & 0xFFu;
      const bool xdirect = ((ud.y >> 24) & 1u) != 0u;
      const int tw = int(G) * VEC;
      const int nst = int(it.se - it.sb);
      unsigned char* stage = s_dyn + st * kTStageBytes;
      T* xs = reinterpret_cast<T*>(stage + kTOffX);
      if (pt == 0 && unit != a.withhold) {   // time-out test: no arrival for the withheld unit
        const int nsl = int((it.hi - it.lo + 31) / 32);
        const uint32_t rb = (it.g1 - it.g0) * uint32_t(kGroup);
        const bool rdirect = rb > uint32_t(kTRecBytes);
        const uint32_t mb = uint32_t(nsl) * kSliceMap;
        constexpr int64_t es_aux = PASS_A ? 8 : 4;
        const int64_t clo = (int64_t(it.slice0) * 4) & ~int64_t(15);
        const int64_t chi = ((int64_t(it.slice0) + nsl + 1) * 4 + 15) & ~int64_t(15);
        const int64_t alo = (int64_t(it.lo) * es_aux) & ~int64_t(15);
        const int64_t ahi = (int64_t(it.hi) * es_aux + 15) & ~int64_t(15);
        TMeta m;
        m.it = it;
        m.col0 = col0;
        m.G = G;
        m.flags = (rdirect ? 1u : 0u) | (xdirect ? 2u : 0u);
        m.coff = int((int64_t(it.slice0) * 4 - clo) / 4);
        m.aoff = int((int64_t(it.lo) * es_aux - alo) / es_aux);
        s_meta[st] = m;
        if (!xdirect)
          for (int j = 0; j < int(G); ++j) *reinterpret_cast<uint4*>(xs + nst * tw + j * VEC) = make_uint4(0, 0, 0, 0);
        const uint32_t bytes = (rdirect ? 0u : rb) + mb + uint32_t(chi - clo) + uint32_t(ahi - alo);
        mbar_arrive_tx(&s_full[st], bytes);
        if (!rdirect && rb) bulk_g2s(stage, recg + int64_t(it.g0) * kGroup, rb, &s_full[st]);
        bulk_g2s(stage + kTOffMap, a.smap + int64_t(it.slice0) * 32, mb, &s_full[st]);
        bulk_g2s(stage + kTOffCol, reinterpret_cast<const unsigned char*>(a.col) + clo, uint32_t(chi - clo),
                 &s_full[st]);
        const unsigned char* aux =
            PASS_A ? reinterpret_cast<const unsigned char*>(a.words) : reinterpret_cast<const unsigned char*>(a.perm);
        bulk_g2s(stage + kTOffAux, aux + alo, uint32_t(ahi - alo), &s_full[st]);
        issued[st] = i;
      }
      if (!xdirect) {
        // the x rows of the stage range, columns [col0, col0 + tw)
        for (int q = pt; q < nst; q += 32 * kTProd) {
          const int64_t row = PASS_A ? int64_t(it.sb) + q : int64_t(__ldg(a.perm + it.sb + q));
          const T* src = x + row * ld + col0;
          T* dst = xs + q * tw;
          for (int j = 0; j < int(G); ++j) cp_async16(dst + j * VEC, src + j * VEC);
        }
      }
      cp_async_mbar_arrive(&s_full[st]);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's copies land before the CTA exits
  } else {
    // consumers
    for (int64_t i = 0; i < n_my; ++i) {
      const int st = int(i % kTStages);
      if (!mbar_wait(&s_full[st], uint32_t((i / kTStages) & 1), a.spin_limit)) {
        failed = true;
        break;
      }
      const TMeta m = s_meta[st];
      const CItem& it = m.it;
      const int G = int(m.G), tw = G * VEC;
      const int spw = 32 / G;                      // states of a slice taken at once by the warp
      const int tg = lane / G, g = lane - tg * G;
      const bool lane_ok = tg < spw;
      const int col = int(m.col0) + g * VEC;
      const int cvalid = a.ncols - col;
      const unsigned char* stage = s_dyn + st * kTStageBytes;
      const uint32_t* colp = reinterpret_cast<const uint32_t*>(stage + kTOffCol) + m.coff;
      const uint16_t* mapp = reinterpret_cast<const uint16_t*>(stage + kTOffMap);
      const T* xs = reinterpret_cast<const T*>(stage + kTOffX);
      const bool rdirect = (m.flags & 1u) != 0u, xdirect = (m.flags & 2u) != 0u;
      const unsigned char* recb = rdirect ? recg + int64_t(it.g0) * kGroup : stage;
      const int nsl = int((it.hi - it.lo + 31) / 32);
      const int nst = int(it.se - it.sb);
      const bool wide = (it.flags & 1u) != 0u;
      auto gather = [&](int q, T* v) {
        if (!xdirect) {
          load16(xs + q * tw + g * VEC, v);
        } else if (q >= nst) {
#pragma unroll
          for (int u = 0; u < VEC; ++u) v[u] = T(0);
        } else {
          const int64_t row = PASS_A ? int64_t(it.sb) + q : int64_t(__ldg(a.perm + it.sb + q));
          C::load(x + row * ld + col, cvalid, v);
        }
      };
      for (int sl = warp; sl < nsl; sl += kTCons) {
        const uint32_t ga = colp[sl], gz = colp[sl + 1];
        const uint32_t locs = mapp[sl * 32 + lane];
        for (int t0 = 0; t0 < 32; t0 += spw) {
          const int t = t0 + tg;
          const uint16_t loc = uint16_t(__shfl_sync(0xffffffffu, locs, t & 31));
          if (!lane_ok || t >= 32 || loc == kNoState || cvalid <= 0) continue;
          const uint32_t k = it.lo + loc;
          const unsigned char* rp = recb + int64_t(ga - it.g0) * kGroup + t * kLaneBytes;
          Acc<T> acc[VEC];
#pragma unroll
          for (int u = 0; u < VEC; ++u) acc[u].zero();
          if (wide)
            state_sum<T, uint32_t, VEC, 2>(rp, int(gz - ga), a.n_cls, s_c64, s_chi, s_clo, gather, acc);
          else
            state_sum16<T, VEC, 2>(rp, int(gz - ga), nst, a.n_cls, s_c64, s_chi, s_clo, gather, acc);
          T out[VEC];
          if (PASS_A) {
            const uint64_t w = reinterpret_cast<const uint64_t*>(stage + kTOffAux)[m.aoff + loc];
            const uint32_t half = a.n_sites >= 32 ? 0xFFFFFFFFu : ((1u << a.n_sites) - 1u);
            const uint32_t up = uint32_t(w >> a.n_sites), dn = uint32_t(w) & half;
            T xk[VEC], yk[VEC];
            gather(int(k - it.sb), xk);
            C::load(y + int64_t(k) * ld + col, cvalid, yk);
            const Coef<T> dc = diag_of<T>(hp, s_dhi, s_dlo, s_d64, up, dn);
#pragma unroll
            for (int u = 0; u < VEC; ++u) {
              acc[u].fma(dc.hi, dc.lo, xk[u]);
              out[u] = acc[u].value() + yk[u];
            }
            C::store(y + int64_t(k) * ld + col, cvalid, out);
          } else {
            const uint32_t row = reinterpret_cast<const uint32_t*>(stage + kTOffAux)[m.aoff + loc];
#pragma unroll
            for (int u = 0; u < VEC; ++u) out[u] = acc[u].value();
            C::store(y + int64_t(row) * ld + col, cvalid, out);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_empty[st]);
    }
  }
  const int any_failed = __syncthreads_or(failed ? 1 : 0);
  if (any_failed) {
    if (warp == kTCons && lane == 0) {
      // bulk copies still in flight land before the CTA's shared memory is released
      for (int s = 0; s < kTStages; ++s)
        if (issued[s] >= 0) mbar_wait(&s_full[s], uint32_t((issued[s] / kTStages) & 1), a.spin_limit);
    }
    if (threadIdx.x == 0) atomicOr(a.err, 1u);
    __syncthreads();
  }
}

// Work units of a layout for rows of nch chunks of vec elements of es bytes:
// per item the widest tile (<= kTMaxG chunks, balanced over the row) whose
// stage rows plus the zero row fit the x stage; items that do not fit even
// one chunk wide gather from global memory, kTMaxG chunks at a time.
void make_units(const std::vector<uint32_t>& rows, int nch, int vec, int es, std::vector<uint2>& out) {
  out.clear();
  const int gmax = std::min(kTMaxG, nch);
  for (size_t i = 0; i < rows.size(); ++i) {
    const int64_t r = int64_t(rows[i]) + 1;
    int g = gmax;
    while (g > 1 && r * g * vec * es > kTXBytes) --g;
    const bool direct = r * g * vec * es > kTXBytes;
    if (direct) g = gmax;
    const int tiles = (nch + g - 1) / g;
    const int gb = (nch + tiles - 1) / tiles;
    for (int c0 = 0; c0 < nch; c0 += gb) {
      const int gg = std::min(gb, nch - c0);
      out.push_back(make_uint2(uint32_t(i), uint32_t(c0 * vec) | (uint32_t(gg) << 16) | (direct ? (1u << 24) : 0u)));
    }
  }
}

template <typename T>
cudaError_t launch_tiles(mcd_ctx* c, const void* x, void* y, int ncols, int ld) {
  constexpr int VEC = 16 / int(sizeof(T));
  const int nch = (ncols + VEC - 1) / VEC;
  const int smem = kTStages * kTStageBytes + cls_bytes(c);
  static int configured = -1;   // per instantiation
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
      std::vector<uint2> u;
      make_units(cc.stage_rows, nch, VEC, int(sizeof(T)), u);
      void* p = cc.units;
      int64_t cap = cc.units_cap * 8;
      cudaError_t e = grow_bytes(p, cap, int64_t(u.size()) * 8, c->stream);
      cc.units = static_cast<uint2*>(p);
      cc.units_cap = cap / 8;
      if (e == cudaSuccess && !u.empty())
        e = cudaMemcpyAsync(cc.units, u.data(), u.size() * 8, cudaMemcpyHostToDevice, c->stream);
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
    const int grid = int(std::min<int64_t>(a.n_units, device_sms()));
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
  static int configured = -1;   // per instantiation
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

cudaError_t cache_apply_cols(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, bool* used) {
  *used = false;
  const bool f64 = dtype == MCD_F64;
  if (ncols == 1) {
    *used = true;
    return f64 ? launch_strided<double>(c, x, y, ld) : launch_strided<float>(c, x, y, ld);
  }
  const int vec = f64 ? 2 : 4;
  const bool vec_ok = ld % vec == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(y) % 16 == 0 && (ncols + vec - 1) / vec * vec <= 65535;
  if (!vec_ok) return cudaSuccess;
  *used = true;
  return f64 ? launch_tiles<double>(c, x, y, ncols, ld) : launch_tiles<float>(c, x, y, ncols, ld);
}

}  // namespace mcd
