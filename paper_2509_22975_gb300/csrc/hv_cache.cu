// Connection cache of y = H~ x.
//
// The nonzeros of the projected matrix H~ are the hops whose targets are in
// the basis (App. B: targets outside F~ are discarded).  They depend only on
// the basis and the Hamiltonian, so Lanczos (hundreds of H~x with the same
// H~) and band Lanczos (hundreds of H~V) would otherwise enumerate and look
// up the same hops every step.  The first H~x of a basis runs the
// enumeration and the in-block lookup of both passes once (the bond loop and
// masked-popcount sign of the matrix-free kernels; a shared bitmap of the
// block for n <= 16 sites, binary search otherwise) and writes what it finds
// as records:
//   2 bytes  position:14 | sign:1 | amplitude class:1   (<= 2 amplitudes)
//   4 bytes  position:22 | sign:1 | class:9             (otherwise, or an
//            item whose blocks hold more than 16383 states)
// where position is the target's place in its work item's stage range (the
// blocks of the item), so that x of the range can be staged in shared
// memory.  Later H~x stream the records and gather from the staged rows.
//
// Layout of the records: the states of a work item are sorted by their
// number of records (most first; equal counts in position order) and form
// slices of 32; group g of a slice holds, for each lane l, the records
// 4g..4g+3 (2-byte) or 2g, 2g+1 (4-byte) of the lane's state, all ones past
// its last record.  A slice has as many groups as its longest list needs
// (sliced ELL with sorting inside the item), so one warp reads one slice
// with every load aligned, little padding and no per-state offsets.
//
// Per state, the hops are summed per amplitude class and each sum is then
// multiplied by the class's fp64 amplitude (split into two floats for fp32
// vectors); with 2-byte records the class-0 sum is the sum of all hops minus
// the class-1 sum.  The order of every sum is fixed, so results repeat bit
// for bit.
//
// One column (Lanczos): a persistent warp-specialised kernel.  One producer
// thread moves each item's records, lane map, slice offsets, staged x rows
// and per-state words into shared memory with bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier), two stages deep,
// while 12 (fp32 vectors) or 8 (fp64) consumer warps work on the previous
// item from shared memory and only store to global memory.  Pass B reads x in its own (dn-major)
// order from a permuted copy, so that its rows are contiguous, and writes
// its part of y to a scratch vector that pass A streams in.
// Many columns (band Lanczos): CTAs stage x rows of an item with ordinary
// loads and groups of G lanes share a state; with G > 1, pass B reads a
// dn-major copy of X.
#include <atomic>
#include <algorithm>
#include <cstring>
#include <vector>

#include "hv_cache.cuh"

namespace mcd {
namespace {

// streaming one-column kernel: two CTAs per SM, each a producer warp and 12
// (fp32 vectors) or 8 (fp64) consumer warps, two stages
template <typename T>
struct SCfg {
  static constexpr int kCons = sizeof(T) == 4 ? 12 : 8;
  static constexpr int kThreads = 32 * (kCons + 1);
};
constexpr int kSStages = 2;
constexpr int kSRecBytes = 24 * 1024;        // records of one item per stage
constexpr int kSMapBytes = (kCItem / 32) * kSliceMap;
constexpr int kSColBytes = 128;              // slice offsets of an item (17 + alignment)
constexpr int kSXBytes = 16 * 1024 + 32;     // staged x rows per stage (+ alignment slack)
constexpr int kSAuxBytes = kCItem * 8 + 16;  // basis word (pass A) or basis index (pass B) of each state
constexpr int kSAux2Bytes = kCItem * 8 + 16; // pass B's part of y (pass A)
constexpr int kSOffMap = kSRecBytes;
constexpr int kSOffCol = kSOffMap + kSMapBytes;
constexpr int kSOffX = kSOffCol + kSColBytes;
constexpr int kSOffAux = kSOffX + kSXBytes;
constexpr int kSOffAux2 = kSOffAux + kSAuxBytes;
constexpr int kSStageBytes = kSOffAux2 + kSAux2Bytes;
static_assert(kSStageBytes % 16 == 0 && kSOffX % 16 == 0 && kSOffAux % 16 == 0 && kSOffAux2 % 16 == 0,
              "stage buffers on 16-byte boundaries");

// ---- build ------------------------------------------------------------------------

// Enumeration of the found hops of state k (layout position) of an item,
// in bond order; f(j, target position, sign, bond) is called for the j-th
// one.  mn = minor words of the stage range (staged or in global memory).
template <typename F>
__device__ __forceinline__ uint32_t enumerate_state(const CArgs& a, const HamParams& hp, const CItem& it,
                                                    uint32_t sb, const uint32_t* mn, uint32_t k, F f) {
  uint32_t b = it.b0;
  if (it.b1 > it.b0) {   // block of k among b0..b1
    uint32_t lo = it.b0, len = it.b1 - it.b0 + 1;
    while (len > 1) {
      const uint32_t h = len >> 1;
      if (a.blk_off[lo + h] <= k) lo += h;
      len -= h;
    }
    b = lo;
  }
  const int bs = int(a.blk_off[b] - sb), be = int(a.blk_off[b + 1] - sb);
  const uint32_t m = mn[k - sb];
  uint32_t cnt = 0;
  for (int bi = 0; bi < hp.n_bonds; ++bi) {
    const uint32_t mk = hp.bonds[bi].mask;
    if (__popc(m & mk) != 1) continue;
    const int q = find_sorted(mn, bs, be, m ^ mk);
    if (q < 0) continue;
    f(cnt, uint32_t(q), __popc(m & hp.bonds[bi].between) & 1u, bi);
    ++cnt;
  }
  return cnt;
}

__device__ __forceinline__ const uint32_t* stage_minor(const CArgs& a, const CItem& it, uint32_t* s_minor,
                                                       uint32_t& sb) {
  sb = a.blk_off[it.b0];
  const uint32_t se = a.blk_off[it.b1 + 1];
  const int nst = int(se - sb);
  const bool staged = nst <= a.xs_cap;
  __syncthreads();
  if (staged)
    for (int q = threadIdx.x; q < nst; q += blockDim.x) s_minor[q] = a.minor[sb + q];
  __syncthreads();
  return staged ? s_minor : a.minor + sb;
}

// cnt[k] = records of state k; nconn += all of them
__global__ void __launch_bounds__(kCT) cache_count_kernel(const CArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint32_t* s_minor = reinterpret_cast<uint32_t*>(s_dyn);
  unsigned long long nc = 0;
  for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const CItem it = a.items[item];
    uint32_t sb;
    const uint32_t* mn = stage_minor(a, it, s_minor, sb);
    for (uint32_t k = it.lo + threadIdx.x; k < it.hi; k += kCT) {
      const uint32_t c = enumerate_state(a, hp, it, sb, mn, k, [](uint32_t, uint32_t, uint32_t, int) {});
      a.cnt[k] = uint16_t(c);
      nc += c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nc += __shfl_xor_sync(0xffffffffu, nc, o);
  if ((threadIdx.x & 31) == 0 && nc) atomicAdd(a.nconn, nc);
}

// Per item: states sorted by count, most first, equal counts in position
// order (a stable counting sort by one warp: ranks among equal counts by
// __match_any); smap and the groups of each slice.
__global__ void __launch_bounds__(kCT) cache_sort_kernel(const CArgs a) {
  __shared__ uint32_t s_off[kMaxCount];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const CItem it = a.items[item];
    const int ns = int(it.hi - it.lo);
    const int nsl = (ns + 31) / 32;
    const int per = (it.flags & 1u) ? Rec<uint32_t>::kPer : Rec<uint16_t>::kPer;
    __syncthreads();
    for (int i = threadIdx.x; i < kMaxCount; i += kCT) s_off[i] = 0u;
    __syncthreads();
    for (int j = threadIdx.x; j < ns; j += kCT) atomicAdd(&s_off[a.cnt[it.lo + j]], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {   // exclusive offsets, largest count first
      uint32_t run = 0;
      for (int c = kMaxCount - 1; c >= 0; --c) {
        const uint32_t v = s_off[c];
        s_off[c] = run;
        run += v;
      }
    }
    __syncthreads();
    uint16_t* sm = a.smap_out + int64_t(it.slice0) * 32;
    if (warp == 0) {
      for (int base = 0; base < ns; base += 32) {
        const int j = base + lane;
        const uint32_t c = j < ns ? a.cnt[it.lo + j] : uint32_t(kMaxCount);   // kMaxCount: no state
        const uint32_t peers = __match_any_sync(0xffffffffu, c);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        const uint32_t p = c < uint32_t(kMaxCount) ? s_off[c] + rank : 0u;
        __syncwarp();
        if (c < uint32_t(kMaxCount) && (peers >> lane) == 1u) s_off[c] += __popc(peers);   // highest peer
        __syncwarp();
        if (j < ns) sm[p] = uint16_t(j);
      }
    }
    __syncthreads();
    for (int p = ns + threadIdx.x; p < nsl * 32; p += kCT) sm[p] = kNoState;
    __syncthreads();
    for (int sl = threadIdx.x; sl < nsl; sl += kCT) {
      const uint32_t c = a.cnt[it.lo + sm[sl * 32]];   // the slice's first state has the most records
      a.wid[it.slice0 + sl] = (c + per - 1) / per;
    }
  }
}

template <typename R>
__device__ __forceinline__ void write_state(const CArgs& a, const HamParams& hp, const uint16_t* s_cls,
                                            const CItem& it, uint32_t sb, const uint32_t* mn, int64_t s,
                                            int lane, uint16_t loc) {
  constexpr int kRow = kGroup / int(sizeof(R));
  const uint32_t g0 = a.col[s];
  const int width = int(a.col[s + 1] - g0) * Rec<R>::kPer;
  R* base = static_cast<R*>(a.rec) + int64_t(g0) * kRow + lane * Rec<R>::kPer;
  auto put = [&](uint32_t j, uint32_t r) {
    if (int(j) < width) base[int64_t(j / Rec<R>::kPer) * kRow + (j % Rec<R>::kPer)] = R(r);
  };
  uint32_t cnt = 0;
  if (loc != kNoState)
    cnt = enumerate_state(a, hp, it, sb, mn, it.lo + loc, [&](uint32_t j, uint32_t q, uint32_t ng, int bi) {
      put(j, Rec<R>::make(q, ng, s_cls[bi]));
    });
  for (int j = int(cnt); j < width; ++j) put(uint32_t(j), Rec<R>::kSent);
}

__global__ void __launch_bounds__(kCT) cache_write_kernel(const CArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint32_t* s_minor = reinterpret_cast<uint32_t*>(s_dyn);
  __shared__ uint16_t s_cls[kMaxBonds];
  for (int i = threadIdx.x; i < hp.n_bonds; i += kCT) s_cls[i] = a.bond_cls[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const CItem it = a.items[item];
    uint32_t sb;
    const uint32_t* mn = stage_minor(a, it, s_minor, sb);
    const int nsl = int((it.hi - it.lo + 31) / 32);
    for (int sl = warp; sl < nsl; sl += kCWarps) {
      const int64_t s = int64_t(it.slice0) + sl;
      const uint16_t loc = a.smap[s * 32 + lane];
      if (it.flags & 1u)
        write_state<uint32_t>(a, hp, s_cls, it, sb, mn, s, lane, loc);
      else
        write_state<uint16_t>(a, hp, s_cls, it, sb, mn, s, lane, loc);
    }
  }
}

// Builds for n_sites <= 16: the in-block lookup by a shared bitmap of the
// block's minor words (bit per word value, with the stage position of the
// first set bit of each 32-bit word), block by block; same bond order, so
// the same records as the binary-search build.
template <typename F>
__device__ __forceinline__ uint32_t enumerate_bm(const HamParams& hp, const uint2* bm, uint32_t m, F f) {
  uint32_t cnt = 0;
  for (int bi = 0; bi < hp.n_bonds; ++bi) {
    const uint32_t mk = hp.bonds[bi].mask;
    if (__popc(m & mk) != 1) continue;
    const uint32_t m2 = m ^ mk;
    const uint2 w = bm[m2 >> 5];
    const uint32_t sh = m2 & 31u;
    if (!((w.x >> sh) & 1u)) continue;
    f(cnt, w.y + __popc(w.x & ((1u << sh) - 1u)), __popc(m & hp.bonds[bi].between) & 1u, bi);
    ++cnt;
  }
  return cnt;
}

template <typename R>
__device__ __forceinline__ void write_bm(const CArgs& a, const HamParams& hp, const uint16_t* s_cls, const uint2* bm,
                                        const CItem& it, uint32_t m, int slot) {
  constexpr int kRow = kGroup / int(sizeof(R));
  const int64_t s = int64_t(it.slice0) + slot / 32;
  const uint32_t g0 = a.col[s];
  const int width = int(a.col[s + 1] - g0) * Rec<R>::kPer;
  R* base = static_cast<R*>(a.rec) + int64_t(g0) * kRow + (slot % 32) * Rec<R>::kPer;
  auto put = [&](uint32_t j, uint32_t r) {
    if (int(j) < width) base[int64_t(j / Rec<R>::kPer) * kRow + (j % Rec<R>::kPer)] = R(r);
  };
  const uint32_t cnt = enumerate_bm(hp, bm, m, [&](uint32_t j, uint32_t q, uint32_t ng, int bi) {
    put(j, Rec<R>::make(q, ng, s_cls[bi]));
  });
  for (int j = int(cnt); j < width; ++j) put(uint32_t(j), Rec<R>::kSent);
}

// WRITE = false: cnt[k] and nconn; WRITE = true: the records (the slots of
// an item's states from the inverse of its lane map; padding of empty slots
// by the lanes that own them)
template <bool WRITE>
__global__ void __launch_bounds__(kCT) cache_bm_kernel(const CArgs a, const HamParams hp, int nw) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  uint2* bm = reinterpret_cast<uint2*>(s_dyn);   // [nw]
  __shared__ uint16_t s_cls[kMaxBonds];
  __shared__ uint16_t s_slot[kCItem];
  for (int i = threadIdx.x; i < nw; i += kCT) bm[i] = make_uint2(0u, 0u);
  for (int i = threadIdx.x; i < hp.n_bonds; i += kCT) s_cls[i] = a.bond_cls[i];
  unsigned long long nc = 0;
  for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const CItem it = a.items[item];
    const uint32_t sb = it.sb;
    const int nsl = int((it.hi - it.lo + 31) / 32);
    const bool wide = (it.flags & 1u) != 0u;
    __syncthreads();
    if (WRITE) {
      for (int p = threadIdx.x; p < nsl * 32; p += kCT) {
        const uint16_t loc = a.smap[int64_t(it.slice0) * 32 + p];
        if (loc != kNoState) {
          s_slot[loc] = uint16_t(p);
        } else {   // an empty slot: its lane's records are all padding
          const int64_t s = int64_t(it.slice0) + p / 32;
          const uint32_t g0 = a.col[s], g1 = a.col[s + 1];
          for (uint32_t g = g0; g < g1; ++g)
            *reinterpret_cast<uint2*>(static_cast<unsigned char*>(a.rec) + int64_t(g) * kGroup + (p % 32) * kLaneBytes) =
                make_uint2(~0u, ~0u);
        }
      }
    }
    for (uint32_t b = it.b0; b <= it.b1; ++b) {
      const uint32_t bs = a.blk_off[b], be = a.blk_off[b + 1];
      __syncthreads();
      for (uint32_t q = threadIdx.x; q < be - bs; q += kCT) {
        const uint32_t d = a.minor[bs + q];
        atomicOr(&bm[d >> 5].x, 1u << (d & 31));
        if (q == 0 || (a.minor[bs + q - 1] >> 5) != (d >> 5)) bm[d >> 5].y = bs - sb + q;
      }
      __syncthreads();
      const uint32_t klo = bs > it.lo ? bs : it.lo, khi = be < it.hi ? be : it.hi;
      for (uint32_t k = klo + threadIdx.x; k < khi; k += kCT) {
        const uint32_t m = a.minor[k];
        if (WRITE) {
          if (wide)
            write_bm<uint32_t>(a, hp, s_cls, bm, it, m, s_slot[k - it.lo]);
          else
            write_bm<uint16_t>(a, hp, s_cls, bm, it, m, s_slot[k - it.lo]);
        } else {
          const uint32_t c = enumerate_bm(hp, bm, m, [](uint32_t, uint32_t, uint32_t, int) {});
          a.cnt[k] = uint16_t(c);
          nc += c;
        }
      }
      __syncthreads();
      for (uint32_t q = threadIdx.x; q < be - bs; q += kCT) bm[a.minor[bs + q] >> 5].x = 0u;
    }
  }
  if (!WRITE) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nc += __shfl_xor_sync(0xffffffffu, nc, o);
    if ((threadIdx.x & 31) == 0 && nc) atomicAdd(a.nconn, nc);
  }
}

// g0, g1 of every item from the slice offsets
__global__ void item_groups_kernel(CItem* items, int64_t n_items, const uint32_t* col) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  CItem& it = items[i];
  it.g0 = col[it.slice0];
  it.g1 = col[it.slice0 + (it.hi - it.lo + 31) / 32];
}

// ---- apply --------------------------------------------------------------------------

// One item of the streaming kernel, for the calling consumer warp: its
// slices warp, warp + kCons, ...  colp = slice offsets from the item's first
// slice, recp = the item's first record group, mapp = lane map, xs = x row
// of stage position 0, wp / pp / ybp = basis word, basis index and pass B's
// part of y of the item's states (by position from it.lo).  DOT: the
// thread's part of <x, y> as an unevaluated sum dh + dl (fp32 vectors: the
// exact products summed with compensation, since GB300's fp64 pipe is too
// narrow for a per-state fp64 product).
template <typename T, bool PASS_A, bool DOT>
__device__ __forceinline__ void consume_item(const CArgs& a, const HamParams& hp, const CItem& it, uint32_t sb,
                                             const uint32_t* colp, const unsigned char* recp, const uint16_t* mapp,
                                             const T* xs, const uint64_t* wp, const uint32_t* pp, const T* ybp,
                                             const double* c64, const float* chi, const float* clo,
                                             const float* dhi, const float* dlo, const double* d64, T& dh, T& dl,
                                             int rot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t half = a.n_sites >= 32 ? 0xFFFFFFFFu : ((1u << a.n_sites) - 1u);
  const int nsl = int((it.hi - it.lo + 31) / 32);
  const uint32_t g0 = colp[0];
  const bool wide = (it.flags & 1u) != 0u;
  T* __restrict__ y = static_cast<T*>(a.y);
  T* __restrict__ yb = static_cast<T*>(a.yb);
  // Slices, longest first (the states are sorted by record count), go to the
  // consumer warps in serpentine order: pass p of kCons slices runs forwards
  // for even p and backwards for odd p, so the warps that take a second slice
  // are those with the shortest first one; the order is rotated by rot, which
  // changes from item to item, so that the extra slices fall on other warps.
  const int wpos = (warp + SCfg<T>::kCons - rot) % SCfg<T>::kCons;
  for (int pass = 0;; ++pass) {
    const int sl = serp_slice(pass, wpos, SCfg<T>::kCons);
    if (sl >= nsl) break;
    const uint16_t loc = mapp[sl * 32 + lane];
    if (loc == kNoState) continue;
    const uint32_t k = it.lo + loc;
    const uint32_t ga = colp[sl], gz = colp[sl + 1];
    const unsigned char* rp = recp + int64_t(ga - g0) * kGroup + lane * kLaneBytes;
    Acc<T> acc[1];
    acc[0].zero();
    auto gather = [&](int q, T* v) { v[0] = xs[q]; };
    if (wide)
      state_sum<T, uint32_t, 1, 4>(rp, int(gz - ga), a.n_cls, c64, chi, clo, gather, acc);
    else
      state_sum<T, uint16_t, 1, 4>(rp, int(gz - ga), a.n_cls, c64, chi, clo, gather, acc);
    if (PASS_A) {
      const uint64_t w = wp[loc];
      const uint32_t up = uint32_t(w >> a.n_sites), dn = uint32_t(w) & half;
      const T xk = xs[k - sb];
      const Coef<T> dc = diag_of<T>(hp, dhi, dlo, d64, up, dn);
      acc[0].fma(dc.hi, dc.lo, xk);
      const T out = acc[0].value() + ybp[loc];
      y[k] = out;
      if constexpr (DOT) {
        if constexpr (sizeof(T) == 4) {
          const T p = xk * out;
          const T pe = fmaf(xk, out, -p);           // exact error of the product
          const T ssum = dh + p, bb = ssum - dh;    // two-sum of the running hi part and p
          dl += (dh - (ssum - bb)) + (p - bb) + pe;
          dh = ssum;
        } else {
          dh = fma(xk, out, dh);
        }
      }
    } else {
      yb[pp[loc]] = acc[0].value();
    }
  }
}

// Fixed-order <x, y> of pass A: CTA partials, then the last CTA sums them.
template <int kWarps>
__device__ __forceinline__ void dot_reduce(const CArgs& a, double dot_acc, double* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot_acc += __shfl_xor_sync(0xffffffffu, dot_acc, o);
  __syncthreads();
  if (lane == 0) s_red[warp] = dot_acc;
  __syncthreads();
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kWarps; ++w) sum += s_red[w];
    a.dot_partials[blockIdx.x] = sum;
    __threadfence();
    const unsigned tk = atomicAdd(a.ticket, 1u);
    s_last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) {
    double sum = 0.0;
    for (int i = threadIdx.x; i < int(gridDim.x); i += blockDim.x) sum += __ldcg(a.dot_partials + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __syncthreads();
    if (lane == 0) s_red[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < kWarps; ++w) tot += s_red[w];
      *a.dot_out = tot;
      *a.ticket = 0u;
    }
  }
}

// One column, persistent and warp-specialised (see the top of the file).
// Items of this CTA: blockIdx.x + i gridDim.x.  Stage i % kSStages holds
// item i: its records, lane map, slice offsets, the x rows of its stage
// range and, per state, the basis word and pass B's part of y (pass A) or
// the basis index (pass B), each copied as whole aligned 16-byte units that
// cover the range.  full[st] completes when the bytes have landed (or the
// producer has marked the item direct: consumers then read global memory),
// empty[st] when the SCfg<T>::kCons consumer warps are done with it.
template <typename T, bool PASS_A, bool DOT>
__global__ void __launch_bounds__(SCfg<T>::kThreads, 2) hv_stream_kernel(const CArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ __align__(8) uint64_t s_full[kSStages], s_empty[kSStages];
  __shared__ int s_direct[kSStages], s_xoff[kSStages], s_coff[kSStages], s_aoff[kSStages], s_boff[kSStages];
  __shared__ CItem s_item[kSStages];
  __shared__ int64_t s_idx[kSStages];   // work item in each stage (-1: no more items)
  __shared__ uint32_t s_sb[kSStages];
  __shared__ float s_dhi[kMaxSites + 1], s_dlo[kMaxSites + 1];
  __shared__ double s_d64[kMaxSites + 1];
  __shared__ double s_red[SCfg<T>::kCons + 1];
  double* s_c64 = reinterpret_cast<double*>(s_dyn + kSStages * kSStageBytes);
  float* s_chi = reinterpret_cast<float*>(s_c64 + a.n_cls);
  float* s_clo = s_chi + a.n_cls;
  for (int i = threadIdx.x; i < a.n_cls; i += SCfg<T>::kThreads) {
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
    for (int s = 0; s < kSStages; ++s) {
      mbar_init(&s_full[s], 1);
      mbar_init(&s_empty[s], SCfg<T>::kCons);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* __restrict__ xg = static_cast<const T*>(PASS_A ? a.x : a.xb);   // rows in layout order
  T dh = T(0), dl = T(0);   // this thread's part of <x, y> (consumers)
  const T* __restrict__ yb = static_cast<const T*>(a.yb);                    // pass B's part of y
  const unsigned char* recg = static_cast<const unsigned char*>(a.rec);
  bool failed = false;
  int64_t issued[kSStages];   // producer: last item index issued into each stage (-1 none)
  for (int s = 0; s < kSStages; ++s) issued[s] = -1;

  if (warp == SCfg<T>::kCons) {
    // producer: one thread takes the CTA's work items (one ahead: the next
    // item's descriptor loads while this one is issued) and issues their
    // copies; past the last item it hands the consumers an end marker.  With
    // <x, y> the items are blockIdx.x + i gridDim.x (the CTA partials then have
    // a fixed order); without, they are claimed from the launch's counter, so
    // CTAs that drew short items take more of them.
    if (lane == 0) {
      int64_t claims = 0;
      auto claim = [&]() -> int64_t {
        if constexpr (DOT) return int64_t(blockIdx.x) + (claims++) * int64_t(gridDim.x);
        return int64_t(atomicAdd(a.sched, 1u));
      };
      CItem nxt{};
      int64_t idx_next = claim();
      if (idx_next < a.n_items) nxt = a.items[idx_next];
      for (int64_t i = 0;; ++i) {
        const int st = int(i % kSStages);
        const CItem it = nxt;
        const int64_t idx = idx_next;
        if (idx < a.n_items) {
          idx_next = claim();
          if (idx_next < a.n_items) nxt = a.items[idx_next];
        }
        if (!mbar_wait(&s_empty[st], uint32_t((i / kSStages) & 1) ^ 1u, a.spin_limit)) {
          failed = true;
          break;
        }
        if (idx >= a.n_items) {
          s_idx[st] = -1;
          mbar_arrive(&s_full[st]);
          break;
        }
        s_idx[st] = idx;
        const uint32_t sb = it.sb, se = it.se;
        const int nsl = int((it.hi - it.lo + 31) / 32);
        const uint32_t g0 = it.g0, g1 = it.g1;
        const uint32_t rb = (g1 - g0) * uint32_t(kGroup);
        const uint32_t mb = uint32_t(nsl) * kSliceMap;
        // 16-byte units covering [first, last) elements of size es
        auto span = [](int64_t first, int64_t last, int64_t es, int64_t& lo16, int64_t& hi16) {
          lo16 = (first * es) & ~int64_t(15);
          hi16 = (last * es + 15) & ~int64_t(15);
        };
        int64_t xlo, xhi, clo, chi, alo, ahi, blo = 0, bhi = 0;
        span(sb, se, sizeof(T), xlo, xhi);
        span(it.slice0, int64_t(it.slice0) + nsl + 1, 4, clo, chi);
        if (PASS_A) {
          span(it.lo, it.hi, 8, alo, ahi);            // basis words
          span(it.lo, it.hi, sizeof(T), blo, bhi);    // pass B's part of y
        } else {
          span(it.lo, it.hi, 4, alo, ahi);            // basis index of each position
        }
        // direct: the records do not fit (everything from global memory); x_out:
        // only the x rows do not (they are gathered from global memory)
        const bool direct = rb > uint32_t(kSRecBytes);
        const bool x_out = xhi - xlo > int64_t(kSXBytes) || xhi > a.x_bytes;
        s_item[st] = it;
        s_sb[st] = sb;
        s_direct[st] = direct ? 1 : (x_out ? 2 : 0);
        s_xoff[st] = int((int64_t(sb) * int64_t(sizeof(T)) - xlo) / int64_t(sizeof(T)));
        s_coff[st] = int((int64_t(it.slice0) * 4 - clo) / 4);
        s_aoff[st] = int((int64_t(it.lo) * (PASS_A ? 8 : 4) - alo) / (PASS_A ? 8 : 4));
        s_boff[st] = int((int64_t(it.lo) * int64_t(sizeof(T)) - blo) / int64_t(sizeof(T)));
        unsigned char* stage = s_dyn + st * kSStageBytes;
        const uint32_t bytes = direct ? 0u
                                      : rb + mb + uint32_t(chi - clo) + (x_out ? 0u : uint32_t(xhi - xlo)) +
                                            uint32_t(ahi - alo) + uint32_t(bhi - blo);
        if (idx == a.withhold) {
          // time-out test: no arrival and no copy for this item, so the
          // waits on its stage run out (nothing is in flight for it)
        } else if (bytes == 0u) {
          mbar_arrive(&s_full[st]);
        } else {
          mbar_arrive_tx(&s_full[st], bytes);
          if (rb) bulk_g2s(stage, recg + int64_t(g0) * kGroup, rb, &s_full[st]);
          bulk_g2s(stage + kSOffMap, a.smap + int64_t(it.slice0) * 32, mb, &s_full[st]);
          bulk_g2s(stage + kSOffCol, reinterpret_cast<const unsigned char*>(a.col) + clo, uint32_t(chi - clo),
                   &s_full[st]);
          if (!x_out && xhi > xlo)
            bulk_g2s(stage + kSOffX, reinterpret_cast<const unsigned char*>(xg) + xlo, uint32_t(xhi - xlo),
                     &s_full[st]);
          const unsigned char* aux =
              PASS_A ? reinterpret_cast<const unsigned char*>(a.words) : reinterpret_cast<const unsigned char*>(a.perm);
          bulk_g2s(stage + kSOffAux, aux + alo, uint32_t(ahi - alo), &s_full[st]);
          if (PASS_A)
            bulk_g2s(stage + kSOffAux2, reinterpret_cast<const unsigned char*>(yb) + blo, uint32_t(bhi - blo),
                     &s_full[st]);
        }
        issued[st] = i;
      }
    }
  } else {
    // consumers: the items of the stages in turn until the end marker
    for (int64_t i = 0;; ++i) {
      const int st = int(i % kSStages);
      if (!mbar_wait(&s_full[st], uint32_t((i / kSStages) & 1), a.spin_limit)) {
        failed = true;
        break;
      }
      const int64_t idx = s_idx[st];
      if (idx < 0) break;
      const int rot = int((idx * 4) % SCfg<T>::kCons);
      const CItem it = s_item[st];
      const unsigned char* stage = s_dyn + st * kSStageBytes;
      if (s_direct[st] == 0) {   // every array of the item in the stage: shared-memory loads
        const uint32_t* colp = reinterpret_cast<const uint32_t*>(stage + kSOffCol) + s_coff[st];
        consume_item<T, PASS_A, DOT>(a, hp, it, s_sb[st], colp, stage,
                                     reinterpret_cast<const uint16_t*>(stage + kSOffMap),
                                     reinterpret_cast<const T*>(stage + kSOffX) + s_xoff[st],
                                     reinterpret_cast<const uint64_t*>(stage + kSOffAux) + s_aoff[st],
                                     reinterpret_cast<const uint32_t*>(stage + kSOffAux) + s_aoff[st],
                                     reinterpret_cast<const T*>(stage + kSOffAux2) + s_boff[st], s_c64, s_chi,
                                     s_clo, s_dhi, s_dlo, s_d64, dh, dl, rot);
      } else if (s_direct[st] == 2) {   // all but the x rows in the stage
        const uint32_t* colp = reinterpret_cast<const uint32_t*>(stage + kSOffCol) + s_coff[st];
        consume_item<T, PASS_A, DOT>(a, hp, it, s_sb[st], colp, stage,
                                     reinterpret_cast<const uint16_t*>(stage + kSOffMap), xg + s_sb[st],
                                     reinterpret_cast<const uint64_t*>(stage + kSOffAux) + s_aoff[st],
                                     reinterpret_cast<const uint32_t*>(stage + kSOffAux) + s_aoff[st],
                                     reinterpret_cast<const T*>(stage + kSOffAux2) + s_boff[st], s_c64, s_chi,
                                     s_clo, s_dhi, s_dlo, s_d64, dh, dl, rot);
      } else {                   // records too large for the stage: global memory
        const uint32_t sb = s_sb[st];
        consume_item<T, PASS_A, DOT>(a, hp, it, sb, a.col + it.slice0, recg + int64_t(it.g0) * kGroup,
                                     a.smap + int64_t(it.slice0) * 32, xg + sb, a.words + it.lo, a.perm + it.lo,
                                     yb + it.lo, s_c64, s_chi, s_clo, s_dhi, s_dlo, s_d64, dh, dl, rot);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_empty[st]);
    }
  }
  const int any_failed = __syncthreads_or(failed ? 1 : 0);
  if (any_failed) {
    if (warp == SCfg<T>::kCons && lane == 0) {
      // copies still in flight land before the CTA's shared memory is released
      for (int s = 0; s < kSStages; ++s)
        if (issued[s] >= 0) mbar_wait(&s_full[s], uint32_t((issued[s] / kSStages) & 1), a.spin_limit);
    }
    if (threadIdx.x == 0) atomicOr(a.err, 1u);
    __syncthreads();
  }
  if constexpr (DOT) {
    dot_reduce<SCfg<T>::kCons + 1>(a, double(dh) + double(dl), s_red);
  } else {
    // the last CTA to finish resets the item counter for the next launch
    __shared__ bool s_last;
    if (threadIdx.x == 0) s_last = atomicAdd(a.sched + 1, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
      a.sched[0] = 0u;
      a.sched[1] = 0u;
    }
  }
}

// x in the layout's order: xb[k] = x[perm[k]] (one column), four positions per
// thread: one 16-byte load of perm, four gathers, 16-byte stores (perm and xb
// start on 16-byte boundaries; the last n % 4 positions one by one)
template <typename T>
__global__ void permute_kernel(const T* __restrict__ x, const uint32_t* __restrict__ perm, int64_t n,
                               T* __restrict__ xb) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nq = n / 4;
  if (q < nq) {
    const uint4 p = __ldg(reinterpret_cast<const uint4*>(perm) + q);
    const T v0 = __ldg(x + p.x), v1 = __ldg(x + p.y), v2 = __ldg(x + p.z), v3 = __ldg(x + p.w);
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float4*>(xb)[q] = make_float4(v0, v1, v2, v3);
    } else {
      reinterpret_cast<double2*>(xb)[2 * q] = make_double2(v0, v1);
      reinterpret_cast<double2*>(xb)[2 * q + 1] = make_double2(v2, v3);
    }
  } else if (q < nq + (n - 4 * nq)) {
    const int64_t k = 4 * nq + (q - nq);
    xb[k] = x[perm[k]];
  }
}

// ---- host ------------------------------------------------------------------------

template <typename P>
cudaError_t grow(P*& p, int64_t& cap, int64_t need, size_t elem, cudaStream_t s) {
  void* q = p;
  int64_t cb = cap * int64_t(elem);
  const cudaError_t e = grow_bytes(q, cb, need * int64_t(elem), s);
  p = static_cast<P*>(q);
  cap = e == cudaSuccess ? cb / int64_t(elem) : 0;
  return e;
}

int sm_count(int dev) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

struct LayoutItems {
  std::vector<CItem> items;
  int64_t n_slices = 0, max_stage = 0;
};

// Work items of a layout: runs of whole blocks of at most kCItem states, or
// pieces of kCItem states of a larger block.  wide_all: every item takes
// 4-byte records; otherwise only items whose stage range is too long for
// 14-bit positions.
void make_items(const std::vector<uint32_t>& off, bool wide_all, LayoutItems& li) {
  li.items.clear();
  li.n_slices = 0;
  li.max_stage = 0;
  const int64_t nblk = int64_t(off.size()) - 1;
  auto add = [&](uint32_t lo, uint32_t hi, uint32_t b0, uint32_t b1) {
    const int64_t stage = int64_t(off[b1 + 1]) - off[b0];
    const bool wide = wide_all || stage > int64_t(Rec<uint16_t>::kMaxStage);
    li.items.push_back(CItem{lo, hi, b0, b1, uint32_t(li.n_slices), wide ? 1u : 0u, off[b0], off[b1 + 1], 0u, 0u});
    li.n_slices += (hi - lo + 31) / 32;
    li.max_stage = std::max(li.max_stage, stage);
  };
  int64_t b = 0;
  while (b < nblk) {
    const uint32_t bsz = off[b + 1] - off[b];
    if (bsz > uint32_t(kCItem)) {
      for (uint32_t p = off[b]; p < off[b + 1]; p += kCItem)
        add(p, std::min<uint32_t>(p + kCItem, off[b + 1]), uint32_t(b), uint32_t(b));
      ++b;
      continue;
    }
    int64_t b1 = b;
    while (b1 + 1 < nblk && off[b1 + 2] - off[b] <= uint32_t(kCItem)) ++b1;
    add(off[b], off[b1 + 1], uint32_t(b), uint32_t(b1));
    b = b1 + 1;
  }
}


int build_layout(mcd_ctx* c, Layout& L, const LayoutItems& li, const std::vector<uint16_t>& bcls,
                 const std::vector<double>& coef, double mem_budget, int64_t& bytes_out) {
  ConnCache& cc = L.cc;
  cudaStream_t s = c->stream;
  const int64_t n_slices = li.n_slices;
  cc.n_items = int64_t(li.items.size());
  cc.n_slices = n_slices;
  cc.max_stage = li.max_stage;
  std::vector<uint2>& rng = c->stage_range[&L == &c->idx.B ? 0 : 1];
  rng.resize(li.items.size());
  for (size_t i = 0; i < li.items.size(); ++i) rng[i] = make_uint2(li.items[i].sb, li.items[i].se);
  cc.units_key = -1;
  std::memset(c->cols_pick, 0, sizeof(c->cols_pick));   // a new basis or Hamiltonian: pick again
  cc.n_cls = int(coef.size());
  const int nc1 = std::max(cc.n_cls, 1);
  cudaError_t e = grow(cc.items, cc.items_cap, cc.n_items, sizeof(CItem), s);
  if (e == cudaSuccess) e = grow(cc.col, cc.col_cap, n_slices + 1 + 4, 4, s);   // + 16 bytes: whole-unit copies
  if (e == cudaSuccess) e = grow(cc.smap, cc.smap_cap, n_slices * 32, 2, s);
  // [c64: nc1 doubles][chi: nc1 floats][clo: nc1 floats][error word]
  if (e == cudaSuccess) e = grow(cc.c64, cc.cls_cap, int64_t(nc1) * 2 + 1, 8, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "cache: tables");
  cc.chi = reinterpret_cast<float*>(cc.c64 + nc1);
  cc.clo = cc.chi + nc1;
  cc.err = reinterpret_cast<unsigned int*>(cc.clo + nc1);
  std::vector<float> hi(coef.size()), lo(coef.size());
  for (size_t i = 0; i < coef.size(); ++i) {
    hi[i] = float(coef[i]);
    lo[i] = float(coef[i] - double(hi[i]));
  }
  uint16_t* d_bcls = nullptr;
  uint16_t* d_cnt = nullptr;
  unsigned long long* d_nc = nullptr;
  uint32_t* wid = nullptr;
  auto release = [&] {
    cudaFreeAsync(d_bcls, s);
    cudaFreeAsync(d_cnt, s);
    cudaFreeAsync(d_nc, s);
    cudaFreeAsync(wid, s);
  };
  e = cudaMemcpyAsync(cc.items, li.items.data(), li.items.size() * sizeof(CItem), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !coef.empty()) {
    e = cudaMemcpyAsync(cc.c64, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cc.chi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cc.clo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(cc.err, 0, 4, s);
  if (e == cudaSuccess && !cc.sched) e = cudaMallocAsync(reinterpret_cast<void**>(&cc.sched), 16, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cc.sched, 0, 16, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_bcls, std::max<size_t>(bcls.size(), 1) * 2, s);
  if (e == cudaSuccess && !bcls.empty())
    e = cudaMemcpyAsync(d_bcls, bcls.data(), bcls.size() * 2, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_cnt, size_t(std::max<int64_t>(L.n, 1)) * 2, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_nc, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_nc, 0, 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&wid, size_t(n_slices + 1) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(wid + n_slices, 0, 4, s);
  CArgs a;
  fill_args(c, L, a);
  a.bond_cls = d_bcls;
  a.cnt = d_cnt;
  a.wid = wid;
  a.smap_out = cc.smap;
  a.nconn = d_nc;
  a.xs_cap = kBuildStageWords;
  const int grid = int(std::min<int64_t>(cc.n_items, int64_t(sm_count(c->device)) * 8));
  const int smem = kBuildStageWords * 4;
  uint32_t total = 0;
  unsigned long long nconn = 0;
  // n_sites <= 16: bitmap lookups (2^n bits of the block's minor words as
  // (bits, first position) pairs); above: binary search in the staged words
  const bool bitmap = c->n <= 16;
  const int nw = c->n >= 5 ? (1 << (c->n - 5)) : 1;
  const int smem_bm = nw * 8;
  if (e == cudaSuccess && cc.n_items > 0) {
    cudaFuncSetAttribute(cache_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(cache_write_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (bitmap)
      cache_bm_kernel<false><<<grid, kCT, smem_bm, s>>>(a, *c->hp, nw);
    else
      cache_count_kernel<<<grid, kCT, smem, s>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    cache_sort_kernel<<<grid, kCT, 0, s>>>(a);
    MCD_LAUNCHED(c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan_u32(c, wid, cc.col, n_slices + 1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, cc.col + n_slices, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nconn, d_nc, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const int64_t bytes = int64_t(total) * kGroup;
  if (e == cudaSuccess && double(bytes) > mem_budget) {
    release();
    cc.failed = 1;
    return MCD_OK;
  }
  if (e == cudaSuccess) e = grow_bytes(cc.rec, cc.rec_cap, bytes, s);
  a.rec = cc.rec;
  if (e == cudaSuccess && cc.n_items > 0 && total > 0) {
    if (bitmap)
      cache_bm_kernel<true><<<grid, kCT, smem_bm, s>>>(a, *c->hp, nw);
    else
      cache_write_kernel<<<grid, kCT, smem, s>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && cc.n_items > 0) {
    item_groups_kernel<<<int((cc.n_items + 255) / 256), 256, 0, s>>>(cc.items, cc.n_items, cc.col);
    MCD_LAUNCHED(c);
    e = cudaGetLastError();
  }
  release();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cc.valid = 0;
    return cuda_fail(c, e, "cache build");
  }
  cc.n_groups = total;
  cc.n_conn = int64_t(nconn);
  cc.valid = 1;
  bytes_out = bytes;
  return MCD_OK;
}

// Records of both layouts for the current basis and Hamiltonian.
int cache_build(mcd_ctx* c) {
  const HamParams& hp = *c->hp;
  // record classes: amplitude classes when there is a class table, else bonds
  std::vector<uint16_t> bcls(size_t(hp.n_bonds));
  std::vector<double> coef;
  if (hp.n_class > 0) {
    int b = 0;
    for (int cl = 0; cl < hp.n_class; ++cl) {
      for (; b < hp.cls_end[cl]; ++b) bcls[size_t(b)] = uint16_t(cl);
      coef.push_back(hp.cls_t[cl]);
    }
  } else {
    for (int b = 0; b < hp.n_bonds; ++b) {
      bcls[size_t(b)] = uint16_t(b);
      coef.push_back(hp.bonds[b].t);
    }
  }
  Layout* Ls[2] = {&c->idx.B, &c->idx.A};
  const bool wide_all = int(coef.size()) > Rec<uint16_t>::kMaxCls;
  LayoutItems li[2];
  int64_t max_stage = 0;
  for (int i = 0; i < 2; ++i) {
    Ls[i]->cc.valid = 0;
    Ls[i]->cc.failed = 0;
    std::vector<uint32_t> off(size_t(Ls[i]->nblk) + 1);
    cudaError_t e = cudaMemcpyAsync(off.data(), Ls[i]->blk_off, off.size() * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cache: block offsets");
    make_items(off, wide_all, li[i]);
    max_stage = std::max(max_stage, li[i].max_stage);
  }
  if (int(coef.size()) > Rec<uint32_t>::kMaxCls || max_stage > int64_t(Rec<uint32_t>::kMaxStage)) {
    for (Layout* L : Ls) L->cc.failed = 1;
    return MCD_OK;
  }
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  // auto: records of both passes within half the free memory
  double budget = c->hv_cache == 2 ? double(freeb) : 0.5 * double(freeb);
  int64_t nconn = 0;
  for (int i = 0; i < 2; ++i) {
    int64_t bytes = 0;
    const int st = build_layout(c, *Ls[i], li[i], bcls, coef, budget, bytes);
    if (st != MCD_OK) return st;
    if (Ls[i]->cc.failed) {
      for (Layout* L : Ls) {
        L->cc.valid = 0;
        L->cc.failed = 1;
      }
      return MCD_OK;
    }
    Ls[i]->cc.rec_bytes = wide_all ? 4 : 2;
    budget -= double(bytes);
    nconn += Ls[i]->cc.n_conn;
  }
  if (c->idx.A.cc.valid && c->idx.B.cc.valid) c->idx.nnz = nconn;
  return MCD_OK;
}


template <typename T>
cudaError_t launch_stream(mcd_ctx* c, const void* x, void* y, double* partials, int max_parts, unsigned int* ticket,
                          double* dot_out) {
  const int smem = kSStages * kSStageBytes + cls_bytes(c);
  static std::atomic<int> configured{-1};   // per instantiation
  if (configured < smem) {
    cudaFuncSetAttribute(hv_stream_kernel<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(hv_stream_kernel<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(hv_stream_kernel<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    configured = smem;
  }
  ConnCache& cb = c->idx.B.cc;
  const int64_t n = c->idx.n;
  // x in dn-major order for pass B and pass B's part of y (padded so that
  // 16-byte copies stay inside)
  const int64_t xb_bytes = (n * int64_t(sizeof(T)) + 15) & ~int64_t(15);
  cudaError_t e = grow_bytes(cb.xb, cb.xb_cap, xb_bytes + 64, c->stream);
  if (e == cudaSuccess) e = grow_bytes(cb.yb, cb.yb_cap, xb_bytes + 64, c->stream);
  if (e != cudaSuccess) return e;
  const int ctas = std::max(1, sm_count(c->device) * (smem <= 110 * 1024 ? 2 : 1));
  for (int pass = 0; pass < 2; ++pass) {
    const Layout& L = pass == 0 ? c->idx.B : c->idx.A;
    CArgs a;
    fill_args(c, L, a);
    a.x = x;
    a.y = y;
    a.xb = cb.xb;
    a.yb = cb.yb;
    a.ncols = 1;
    a.ld = 1;
    // pass A reads the caller's x: only whole 16-byte units inside it
    a.x_bytes = pass == 0 ? xb_bytes
                          : ((reinterpret_cast<uintptr_t>(x) % 16 == 0) ? (n * int64_t(sizeof(T))) & ~int64_t(15) : 0);
    const bool dot = pass == 1 && partials != nullptr;
    if (c->wait_test_item >= 0) {
      a.spin_limit = kTestSpinLimit;
      if (pass == 1) a.withhold = c->wait_test_item;
    }
    a.dot_partials = partials;
    a.ticket = ticket;
    a.dot_out = dot_out;
    a.sched = L.cc.sched;
    int64_t grid = std::min<int64_t>(a.n_items, ctas);
    if (dot) grid = std::min<int64_t>(grid, max_parts);
    if (grid <= 0) {
      if (!dot) continue;
      grid = 1;   // an empty basis still writes <x, y> = 0
    }
    timing_begin(c, pass == 0 ? 0 : 1);
    if (pass == 0) {
      const int64_t threads = n / 4 + n % 4;
      permute_kernel<T><<<int((threads + 255) / 256), 256, 0, c->stream>>>(static_cast<const T*>(x), L.perm, n,
                                                                           static_cast<T*>(cb.xb));
      MCD_LAUNCHED(c);
      hv_stream_kernel<T, false, false><<<int(grid), SCfg<T>::kThreads, smem, c->stream>>>(a, *c->hp);
    } else if (dot) {
      hv_stream_kernel<T, true, true><<<int(grid), SCfg<T>::kThreads, smem, c->stream>>>(a, *c->hp);
    } else {
      hv_stream_kernel<T, true, false><<<int(grid), SCfg<T>::kThreads, smem, c->stream>>>(a, *c->hp);
    }
    MCD_LAUNCHED(c);
    timing_end(c);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  c->wait_test_item = -1;   // the test option applies to one product
  return cudaSuccess;
}


template <typename T>
cudaError_t dispatch(mcd_ctx* c, const void* x, void* y, int ncols, int ld, double* partials, int max_parts,
                     unsigned int* ticket, double* dot_out, bool* used) {
  if (ncols == 1 && ld == 1) {
    *used = true;
    return launch_stream<T>(c, x, y, partials, max_parts, ticket, dot_out);
  }
  if (partials) {   // the fused <x, y> is only formed for contiguous single columns
    *used = false;
    return cudaSuccess;
  }
  return cache_apply_cols(c, x, y, ncols, ld, sizeof(T) == 8 ? MCD_F64 : MCD_F32, used);
}

}  // namespace

void cache_invalidate(Layout& L) {
  L.cc.valid = 0;
  L.cc.failed = 0;
}

void free_cache(Layout& L, cudaStream_t s) {
  ConnCache& cc = L.cc;
  auto f = [s](void* p) { if (p) cudaFreeAsync(p, s); };
  f(cc.items); f(cc.col); f(cc.smap); f(cc.rec); f(cc.c64); f(cc.xb); f(cc.yb); f(cc.xbm); f(cc.units);
  f(cc.sched);
  cc = ConnCache();
}

int cache_apply(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, double* dot_partials,
                int max_parts, unsigned int* ticket, double* dot_out, bool* used) {
  *used = false;
  ConnCache& A = c->idx.A.cc;
  ConnCache& B = c->idx.B.cc;
  if (!(A.valid && B.valid)) {
    if (!(A.failed || B.failed)) {
      const int st = cache_build(c);
      if (st != MCD_OK) return st;
    }
    if (!(A.valid && B.valid)) {
      if (c->hv_cache == 2) return fail(c, MCD_E_INVALID, "connection cache cannot be built for this basis");
      return MCD_OK;
    }
  }
  const cudaError_t e =
      dtype == MCD_F64 ? dispatch<double>(c, x, y, ncols, ld, dot_partials, max_parts, ticket, dot_out, used)
                       : dispatch<float>(c, x, y, ncols, ld, dot_partials, max_parts, ticket, dot_out, used);
  return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "cached H*v launch");
}

int cache_errors(mcd_ctx* c, unsigned int* out) {
  unsigned int v = 0, w = 0;
  cudaError_t e = cudaSuccess;
  if (c->idx.A.cc.err) e = cudaMemcpyAsync(&v, c->idx.A.cc.err, 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && c->idx.B.cc.err)
    e = cudaMemcpyAsync(&w, c->idx.B.cc.err, 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cache error word");
  *out = v | w;
  return MCD_OK;
}

int take_wait_errors(mcd_ctx* c) {
  ConnCache& A = c->idx.A.cc;
  ConnCache& B = c->idx.B.cc;
  if (!A.err && !B.err) return MCD_OK;
  unsigned int v = 0;
  int st = cache_errors(c, &v);
  if (st != MCD_OK || v == 0) return st;
  cudaError_t e = cudaSuccess;
  if (A.err) e = cudaMemsetAsync(A.err, 0, 4, c->stream);
  if (e == cudaSuccess && B.err) e = cudaMemsetAsync(B.err, 0, 4, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "clear wait-error word");
  return fail(c, MCD_E_TIMEOUT, "a bounded wait of the streaming H*v kernel gave up; the product is incomplete");
}

}  // namespace mcd
