// y = H~ x with hash-table lookups inside blocks (any n_sites <= 32).
//
// Same two passes as hv.cu (pass B: dn-major blocks, up-spin hops, writes
// y[perm k]; pass A: up-major blocks, dn-spin hops + diagonal, y[k] +=), and
// the same projection (App. B: a hop whose target is not in the truncated
// basis is dropped).  What differs is the in-block search.  With more than 16
// sites a 2^n-bit bitmap of the block no longer fits in shared memory, and a
// binary search over a block of ~2000 words (the state-weighted mean block of
// a 24-site, 5e7-state basis) costs ~11 dependent shared loads per candidate
// hop, of which ~87% miss.  Here the minor words of a work item are entered
//   - in a membership filter of 32 bits per word (one bit per word, at a
//     hashed position): a target whose bit is clear is absent, which settles
//     ~97% of the absent targets with one shared load, and
//   - in an open-addressing table (linear probing, at most a quarter full)
//     whose 32-bit slot holds (position << 16 | low 16 bits of the word); a
//     hit is confirmed by one load of the stored word.
//
// Work items are runs of whole blocks holding at most `hcap` states; the CTA
// builds their filter and table in shared memory (keys mix the word with the
// block's start, so equal words of different blocks do not collide).  A block
// of more than hcap states is split into chunks of hcap states that share one
// filter (16 bits per word) and one table (at most half full) of that block,
// built once per basis in device memory.
//
// Hops are enumerated from hop groups, the bonds (i, i + s) of one amplitude
// t and one distance s: hg_mask & (m ^ (m >> s)) marks the bonds along which
// the spin word m can hop.  Target m ^ ((1 | 1 << s) << i), fermionic sign
// (-1)^(occupied sites strictly between i and i + s).  One thread per state
// walks a cursor over all groups' candidate hops, two lookups in flight, and
// (single column) moves on to its next state as soon as one is done, so the
// lanes of a warp do not wait for each other at state boundaries.  With
// several columns the found hops of a round of states are listed in shared
// memory and groups of lanes gather their column chunks.
//
// Filter bits and table slots are set by atomics in whatever order threads
// arrive, but a word has one position, so results do not depend on it.
#include <atomic>
#include <algorithm>
#include <vector>

#include "hv_common.cuh"

namespace mcd {
namespace {

constexpr int kHThreads = 256;
constexpr int kHWarps = kHThreads / 32;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kMaxBlockTable = 65534;   // positions must fit 16 bits below 0xFFFF

// multiplicative hash of the word mixed with the block key (top bits = slot)
__device__ __forceinline__ uint32_t hkey(uint32_t m, uint32_t base) {
  return (m ^ (base * 0x9E3779B9u)) * 0x85EBCA6Bu;
}

template <bool GLOBAL>
__device__ __forceinline__ uint32_t ld32(const uint32_t* p) {
  if (GLOBAL) return __ldg(p);
  return *p;
}

// position p in [lo, hi) with words[p] == m2, or -1
template <bool GLOBAL>
__device__ __forceinline__ int hfind(const uint32_t* tab, int log2p, const uint32_t* words, uint32_t m2,
                                     uint32_t base, int lo, int hi) {
  const uint32_t msk = (1u << log2p) - 1u;
  uint32_t s = hkey(m2, base) >> (32 - log2p);
  const uint32_t fp = m2 & 0xFFFFu;
  for (uint32_t it = 0; it <= msk; ++it) {
    const uint32_t e = ld32<GLOBAL>(tab + s);
    if (e == kEmpty) return -1;
    if ((e & 0xFFFFu) == fp) {
      const int p = int(e >> 16);
      if (p >= lo && p < hi && ld32<GLOBAL>(words + p) == m2) return p;
    }
    s = (s + 1u) & msk;
  }
  return -1;
}

// second multiplicative hash (top bits = filter bit)
__device__ __forceinline__ uint32_t fkey(uint32_t m, uint32_t base) {
  return (m ^ (base * 0x7FEB352Du)) * 0x846CA68Bu;
}

__device__ __forceinline__ void finsert(uint32_t* flt, int log2f, uint32_t m, uint32_t base) {
  const uint32_t bit = fkey(m, base) >> (32 - log2f);
  atomicOr(flt + (bit >> 5), 1u << (bit & 31u));
}

template <bool GLOBAL>
__device__ __forceinline__ bool fhas(const uint32_t* flt, int log2f, uint32_t m, uint32_t base) {
  const uint32_t bit = fkey(m, base) >> (32 - log2f);
  return (ld32<GLOBAL>(flt + (bit >> 5)) >> (bit & 31u)) & 1u;
}

__device__ __forceinline__ void hinsert(uint32_t* tab, int log2p, uint32_t m, uint32_t base, int p) {
  const uint32_t msk = (1u << log2p) - 1u;
  uint32_t s = hkey(m, base) >> (32 - log2p);
  const uint32_t e = (uint32_t(p) << 16) | (m & 0xFFFFu);
  for (uint32_t it = 0; it <= msk; ++it) {   // the table is at most half full
    if (atomicCAS(tab + s, kEmpty, e) == kEmpty) return;
    s = (s + 1u) & msk;
  }
}

// tables of the blocks above the item size, one CTA per block
__global__ void block_tables_kernel(const Layout L, const uint32_t* big, int n_big, uint32_t* htab,
                                    uint32_t* hflt, const HItem* items) {
  const int bi = blockIdx.x;
  if (bi >= n_big) return;
  const HItem it = items[big[bi]];
  const int bs = int(L.blk_off[it.b0]), be = int(L.blk_off[it.b0 + 1]);
  for (int p = threadIdx.x; p < be - bs; p += blockDim.x) {
    const uint32_t m = L.minor[bs + p];
    hinsert(htab + it.tab_off, int(it.log2p), m, 0u, p);
    finsert(hflt + it.flt_off, int(it.log2f), m, 0u);
  }
}

// Lookup context of one state: where its block's words and table live.
struct Where {
  const uint32_t* flt;     // membership filter of 2^log2f bits
  int log2f;
  const uint32_t* tab;
  const uint32_t* words;   // words[p] = minor word of layout position pbase + p
  int log2p;               // kHashSearch: binary search of words[lo, hi)
  uint32_t base;           // block key
  int lo, hi;              // the block's positions
  int pbase;               // layout position of p = 0
};

// Lookup modes: 0 = filter and table in shared memory (small items);
// 1 = filter copied to shared memory, table in device memory (chunks of a
// tabled block whose filter fits); 2 = both in device memory, or binary
// search when the block has no table.
template <int MODE>
__device__ __forceinline__ int lookup(const Where& w, uint32_t m2) {
  if (MODE == 0) {
    if (!fhas<false>(w.flt, w.log2f, m2, w.base)) return -1;
    return hfind<false>(w.tab, w.log2p, w.words, m2, w.base, w.lo, w.hi);
  }
  if (MODE == 1) {
    if (!fhas<false>(w.flt, w.log2f, m2, 0u)) return -1;
    return hfind<true>(w.tab, w.log2p, w.words, m2, w.base, w.lo, w.hi);
  }
  if (w.log2p == int(kHashSearch)) {
    int len = w.hi - w.lo;
    const uint32_t* p = w.words + w.lo;
    if (len <= 0) return -1;
    while (len > 1) {
      const int half = len >> 1;
      if (__ldg(p + half) <= m2) p += half;
      len -= half;
    }
    return (__ldg(p) == m2) ? int(p - w.words) : -1;
  }
  if (!fhas<true>(w.flt, w.log2f, m2, 0u)) return -1;
  return hfind<true>(w.tab, w.log2p, w.words, m2, w.base, w.lo, w.hi);
}

__device__ __forceinline__ uint32_t between_bits(int i, int s) {
  return ((1u << (s - 1)) - 1u) << (i + 1);   // sites i+1 .. i+s-1
}

template <typename T, int VEC, bool PASS_A>
struct Rows {
  const T* x;
  const T* xs;       // staged single-column x of the item (nullptr: from global)
  const uint32_t* perm;
  int ld;
  __device__ __forceinline__ void fetch(const Where& w, int q, int col, int cvalid, T* v) const {
    if (VEC == 1 && xs) {
      v[0] = xs[q];
    } else {
      const int pos = w.pbase + q;
      const int64_t row = PASS_A ? int64_t(pos) : int64_t(__ldg(perm + pos));
      ChunkOf<T, VEC>::load(x + row * ld + col, cvalid, v);
    }
  }
};

template <typename T>
__device__ __forceinline__ T coef_hi(const float* hi, const double* t, int g) {
  return sizeof(T) == 4 ? T(hi[g]) : T(t[g]);
}
template <typename T>
__device__ __forceinline__ T coef_lo(const float* lo, int g) {
  return sizeof(T) == 4 ? T(lo[g]) : T(0);
}

// Cursor over the candidate hops of one spin word: hop groups in order, the
// active bonds of a group in ascending site order.
struct Cursor {
  uint32_t m, act;
  int g, s, nhg;
  __device__ __forceinline__ void start(uint32_t m_, int nhg_, const uint32_t* mask, const int* shift) {
    m = m_;
    nhg = nhg_;
    g = -1;
    act = 0u;
    s = 1;
    next_group(mask, shift);
  }
  __device__ __forceinline__ void next_group(const uint32_t* mask, const int* shift) {
    while (act == 0u && ++g < nhg) {
      s = shift[g];
      act = mask[g] & (m ^ (m >> s));
    }
  }
  __device__ __forceinline__ bool valid() const { return g < nhg; }
  // take the next candidate: site i, distance s, group g
  __device__ __forceinline__ void take(int& i, int& s_, int& g_, const uint32_t* mask, const int* shift) {
    i = __ffs(act) - 1;
    s_ = s;
    g_ = g;
    act &= act - 1u;
    next_group(mask, shift);
  }
};

// shared-memory carve-up of an item: table, words, block offsets and indices
struct ItemSmem {
  uint32_t* flt;
  uint32_t* tab;
  uint32_t* wds;
  uint16_t* boff;
  uint16_t* bidx;
};

// Build the shared table of a small item (whole blocks [b0, b1)); optionally
// stage the single-column x of its states.
template <typename T, bool PASS_A, bool STAGE>
__device__ __forceinline__ void build_item(const HvArgs& a, const HItem& it, const ItemSmem& sm, T* xs) {
  const Layout& L = a.L;
  const int P1 = 1 << a.hlog2;
  const int S = int(it.s1 - it.s0);
  const int nb = int(it.b1 - it.b0);
  const T* x = static_cast<const T*>(a.x);
  for (int i = threadIdx.x; i < P1; i += blockDim.x) sm.tab[i] = kEmpty;
  for (int i = threadIdx.x; i < (1 << a.flog2) / 32; i += blockDim.x) sm.flt[i] = 0u;
  for (int j = threadIdx.x; j <= nb; j += blockDim.x) sm.boff[j] = uint16_t(__ldg(L.blk_off + it.b0 + j) - it.s0);
  __syncthreads();
  for (int p = threadIdx.x; p < S; p += blockDim.x) {
    const uint32_t k = it.s0 + uint32_t(p);
    const uint32_t m = __ldg(L.minor + k);
    T xv = T(0);
    if (STAGE) xv = __ldg(x + (PASS_A ? int64_t(k) : int64_t(__ldg(L.perm + k))) * a.ld);
    int lo = 0, len = nb;   // block j of p: boff[j] <= p < boff[j + 1]
    while (len > 1) {
      const int half = len >> 1;
      if (int(sm.boff[lo + half]) <= p) lo += half;
      len -= half;
    }
    sm.bidx[p] = uint16_t(lo);
    hinsert(sm.tab, a.hlog2, m, sm.boff[lo], p);
    finsert(sm.flt, a.flog2, m, sm.boff[lo]);
    sm.wds[p] = m;
    if (STAGE) xs[p] = xv;
  }
  __syncthreads();
}

// lookup context of state p of an item
__device__ __forceinline__ Where where_of(const HvArgs& a, const HItem& it, const ItemSmem& sm, bool big, int p,
                                          uint32_t& m, int& b, const uint32_t* sflt = nullptr) {
  const Layout& L = a.L;
  Where w;
  if (big) {
    b = int(it.b0);
    const int bs = int(__ldg(L.blk_off + b));
    w.flt = sflt ? sflt : a.hflt + it.flt_off;
    w.log2f = int(it.log2f);
    w.tab = a.htab + it.tab_off;
    w.words = L.minor + bs;
    w.log2p = int(it.log2p);
    w.base = 0u;
    w.lo = 0;
    w.hi = int(__ldg(L.blk_off + b + 1)) - bs;
    w.pbase = bs;
    m = __ldg(L.minor + it.s0 + p);
  } else {
    const int j = sm.bidx[p];
    b = int(it.b0) + j;
    w.flt = sm.flt;
    w.log2f = a.flog2;
    w.tab = sm.tab;
    w.words = sm.wds;
    w.log2p = a.hlog2;
    w.lo = sm.boff[j];
    w.hi = sm.boff[j + 1];
    w.base = uint32_t(w.lo);
    w.pbase = int(it.s0);
    m = sm.wds[p];
  }
  return w;
}

template <typename T>
__device__ __forceinline__ Coef<T> diag_of(const HamParams& hp, const float* dhi, const float* dlo,
                                           const double* d64, uint32_t major, uint32_t m) {
  Coef<T> dc;
  if (hp.uniform) {
    const int nu = __popc(major & m);
    dc.hi = sizeof(T) == 4 ? T(dhi[nu]) : T(d64[nu]);
    dc.lo = sizeof(T) == 4 ? T(dlo[nu]) : T(0);
  } else {
    dc = diag_coef<T>(hp, major, m);
  }
  return dc;
}

struct HopSmem {
  uint32_t mask[kMaxHopGroups];
  int shift[kMaxHopGroups];
  float hi[kMaxHopGroups], lo[kMaxHopGroups];
  double t[kMaxHopGroups];
  float dhi[kMaxSites + 1], dlo[kMaxSites + 1];
  double d64[kMaxSites + 1];
};

__device__ __forceinline__ void load_hops(const HamParams& hp, HopSmem& H) {
  for (int i = threadIdx.x; i < hp.n_hg; i += blockDim.x) {
    H.mask[i] = hp.hg_mask[i];
    H.shift[i] = hp.hg_shift[i];
    H.hi[i] = hp.hg_hi[i];
    H.lo[i] = hp.hg_lo[i];
    H.t[i] = hp.hg_t[i];
  }
  if (threadIdx.x <= kMaxSites) {
    H.dhi[threadIdx.x] = hp.dtab_hi[threadIdx.x];
    H.dlo[threadIdx.x] = hp.dtab_lo[threadIdx.x];
    H.d64[threadIdx.x] = hp.dtab[threadIdx.x];
  }
}

// per-CTA partial of sum x[k] y[k]; the last CTA to finish sums the partials
// in a fixed order into *dot_out
__device__ __forceinline__ void dot_finish(const HvArgs& a, double dot_acc, double* s_red) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot_acc += __shfl_xor_sync(full, dot_acc, o);
  __syncthreads();
  if (lane == 0) s_red[warp] = dot_acc;
  __syncthreads();
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int i = 0; i < nw; ++i) sum += s_red[i];
    a.dot_partials[blockIdx.x] = sum;
    __threadfence();
    const unsigned t = atomicAdd(a.ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) {
    double sum = 0.0;
    for (int i = threadIdx.x; i < int(gridDim.x); i += blockDim.x) sum += __ldcg(a.dot_partials + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(full, sum, o);
    __syncthreads();
    if (lane == 0) s_red[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int i = 0; i < nw; ++i) tot += s_red[i];
      *a.dot_out = tot;
      *a.ticket = 0u;
    }
  }
}

// Single column, one thread per state.  Each thread streams through the
// candidate hops of its states (two lookups in flight) and moves on to its
// next state as soon as one is done, so lanes do not wait for each other at
// state boundaries; what a state's end needs (y, perm, major) is loaded when
// the state starts.
template <typename T, bool PASS_A, int MODE>
__device__ __forceinline__ void stream_states(const HvArgs& a, const HamParams& hp, const HItem& it,
                                              const ItemSmem& sm, const T* xs, const HopSmem& H,
                                              double& dot_acc) {
  constexpr bool BIG = MODE != 0;
  const Layout& L = a.L;
  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const int S = int(it.s1 - it.s0);
  const Rows<T, 1, PASS_A> R{x, BIG ? nullptr : xs, L.perm, a.ld};
  int p = threadIdx.x;
  if (p >= S) return;
  uint32_t m, major = 0u;
  int b;
  Where w;
  Cursor cur;
  Acc<T> acc;
  T yk = T(0);
  int64_t orow = 0;
  auto begin = [&]() {
    w = where_of(a, it, sm, BIG, p, m, b, MODE == 1 ? sm.tab : nullptr);
    const uint32_t k = it.s0 + uint32_t(p);
    if (PASS_A) {
      yk = y[int64_t(k) * a.ld];
      major = __ldg(L.blk_major + b);
    } else {
      orow = int64_t(__ldg(L.perm + k));
    }
    cur.start(m, hp.n_hg, H.mask, H.shift);
    acc.zero();
  };
  begin();
  for (;;) {
    if (!cur.valid()) {
      if (PASS_A) {
        const uint32_t k = it.s0 + uint32_t(p);
        T xk;
        R.fetch(w, int(k) - w.pbase, 0, 1, &xk);
        const Coef<T> dc = diag_of<T>(hp, H.dhi, H.dlo, H.d64, major, m);
        acc.fma(dc.hi, dc.lo, xk);
        const T out = acc.value() + yk;
        y[int64_t(k) * a.ld] = out;
        dot_acc += double(xk) * double(out);
      } else {
        y[orow * a.ld] = acc.value();
      }
      p += blockDim.x;
      if (p >= S) break;
      begin();
      continue;
    }
    int i1, s1, g1, i2 = 0, s2 = 1, g2 = 0;
    cur.take(i1, s1, g1, H.mask, H.shift);
    const bool two = cur.valid();
    if (two) cur.take(i2, s2, g2, H.mask, H.shift);
    const int q1 = lookup<MODE>(w, m ^ ((1u | (1u << s1)) << i1));
    const int q2 = two ? lookup<MODE>(w, m ^ ((1u | (1u << s2)) << i2)) : -1;
    if (q1 >= 0) {
      T xv;
      R.fetch(w, q1, 0, 1, &xv);
      const bool neg = __popc(m & between_bits(i1, s1)) & 1;
      const T h = coef_hi<T>(H.hi, H.t, g1), l = coef_lo<T>(H.lo, g1);
      acc.fma(neg ? -h : h, neg ? -l : l, xv);
    }
    if (q2 >= 0) {
      T xv;
      R.fetch(w, q2, 0, 1, &xv);
      const bool neg = __popc(m & between_bits(i2, s2)) & 1;
      const T h = coef_hi<T>(H.hi, H.t, g2), l = coef_lo<T>(H.lo, g2);
      acc.fma(neg ? -h : h, neg ? -l : l, xv);
    }
  }
}

// shared-memory carve-up from the argument offsets
__device__ __forceinline__ ItemSmem item_smem_of(const HvArgs& a, unsigned char* base) {
  ItemSmem sm;
  sm.tab = reinterpret_cast<uint32_t*>(base);
  sm.flt = sm.tab + (1 << a.hlog2);
  sm.wds = sm.flt + (1 << a.flog2) / 32;
  sm.boff = reinterpret_cast<uint16_t*>(sm.wds + a.hcap);
  sm.bidx = sm.boff + a.hcap + 2;
  return sm;
}

// Lookup mode of an item (see lookup); mode 1 copies the block's filter to
// the start of the shared item area, which it must fit.
__device__ __forceinline__ int item_mode(const HvArgs& a, const HItem& it, const ItemSmem& sm) {
  if (it.log2p == 0u) return 0;
  if (it.log2p == kHashSearch || ((size_t(1) << it.log2f) / 8) > size_t(a.off_xs)) return 2;
  const int nwords = (1 << it.log2f) / 32;
  const uint32_t* src = a.hflt + it.flt_off;
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) sm.tab[i] = __ldg(src + i);
  __syncthreads();
  return 1;
}

template <typename T, bool PASS_A, bool DOT>
__global__ void __launch_bounds__(kHThreads) hv_hash1_kernel(const HvArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ HopSmem H;
  __shared__ double s_red[kHWarps];
  const ItemSmem sm = item_smem_of(a, s_dyn);
  T* xs = reinterpret_cast<T*>(s_dyn + a.off_xs);
  load_hops(hp, H);
  double dot_acc = 0.0;
  for (int ii = blockIdx.x; ii < a.n_hitems; ii += gridDim.x) {
    const HItem it = a.items[ii];
    __syncthreads();   // the previous item's shared data is no longer read
    const int mode = item_mode(a, it, sm);
    if (mode == 0) {
      build_item<T, PASS_A, true>(a, it, sm, xs);
      stream_states<T, PASS_A, 0>(a, hp, it, sm, xs, H, dot_acc);
    } else if (mode == 1) {
      stream_states<T, PASS_A, 1>(a, hp, it, sm, xs, H, dot_acc);
    } else {
      stream_states<T, PASS_A, 2>(a, hp, it, sm, xs, H, dot_acc);
    }
  }
  if (DOT) dot_finish(a, dot_acc, s_red);
}

constexpr int kHitCap = 24;   // hits per state kept in a round's lists

// Several columns: in rounds of one state per thread, phase 1 streams the
// candidate hops and lists the found ones (position, group and sign byte); phase 2 has G lanes per state gather their VEC-column chunks of the
// listed rows.  A state with more than kHitCap hits has its remaining hits
// found again by its G lanes in phase 2.
template <typename T, int VEC, int G, bool PASS_A, int MODE>
__device__ __forceinline__ void multi_item(const HvArgs& a, const HamParams& hp, const HItem& it,
                                           const ItemSmem& sm, const HopSmem& H, uint32_t* lq, uint8_t* lg,
                                           uint8_t* lcnt) {
  const Layout& L = a.L;
  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const int S = int(it.s1 - it.s0);
  constexpr bool BIG = MODE != 0;
  const uint32_t* sflt = MODE == 1 ? sm.tab : nullptr;
  const Rows<T, VEC, PASS_A> R{x, nullptr, L.perm, a.ld};
  using C = ChunkOf<T, VEC>;
  const int ncols = a.ncols, ld = a.ld;
  const int g = threadIdx.x % G;
  const int group = threadIdx.x / G;
  constexpr int kGroups = kHThreads / G;
  for (int r0 = 0; r0 < S; r0 += kHThreads) {
    // phase 1
    {
      const int p = r0 + int(threadIdx.x);
      int nh = 0;
      if (p < S) {
        uint32_t m;
        int b;
        const Where w = where_of(a, it, sm, BIG, p, m, b, sflt);
        Cursor cur;
        cur.start(m, hp.n_hg, H.mask, H.shift);
        uint32_t* oq = lq + threadIdx.x * kHitCap;
        uint8_t* og = lg + threadIdx.x * kHitCap;
        while (cur.valid()) {
          int i1, s1, g1, i2 = 0, s2 = 1, g2 = 0;
          cur.take(i1, s1, g1, H.mask, H.shift);
          const bool two = cur.valid();
          if (two) cur.take(i2, s2, g2, H.mask, H.shift);
          const int q1 = lookup<MODE>(w, m ^ ((1u | (1u << s1)) << i1));
          const int q2 = two ? lookup<MODE>(w, m ^ ((1u | (1u << s2)) << i2)) : -1;
          if (q1 >= 0) {
            if (nh < kHitCap) {
              oq[nh] = uint32_t(q1);
              og[nh] = uint8_t(g1 | ((__popc(m & between_bits(i1, s1)) & 1) << 7));
            }
            ++nh;
          }
          if (q2 >= 0) {
            if (nh < kHitCap) {
              oq[nh] = uint32_t(q2);
              og[nh] = uint8_t(g2 | ((__popc(m & between_bits(i2, s2)) & 1) << 7));
            }
            ++nh;
          }
        }
      }
      lcnt[threadIdx.x] = uint8_t(nh > kHitCap ? 255 : nh);
    }
    __syncthreads();
    // phase 2
    const int ns = (S - r0 < kHThreads) ? S - r0 : kHThreads;
    for (int t = group; t < ns; t += kGroups) {
      const int p = r0 + t;
      const uint32_t k = it.s0 + uint32_t(p);
      uint32_t m;
      int b;
      const Where w = where_of(a, it, sm, BIG, p, m, b, sflt);
      const int cnt = lcnt[t];
      const int nl = cnt == 255 ? kHitCap : cnt;
      const uint32_t* iq = lq + t * kHitCap;
      const uint8_t* ig = lg + t * kHitCap;
      const int64_t orow = PASS_A ? int64_t(k) : int64_t(__ldg(L.perm + k));
      for (int cb = 0; cb < ncols; cb += G * VEC) {
        const int col = cb + g * VEC;
        const int cvalid = ncols - col;
        if (cvalid <= 0) continue;
        Acc<T> acc[VEC];
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[u].zero();
        for (int h = 0; h < nl; ++h) {
          const uint32_t gg = ig[h];
          const int gi = int(gg & 0x7Fu);
          T ch = coef_hi<T>(H.hi, H.t, gi), cl = coef_lo<T>(H.lo, gi);
          if (gg & 0x80u) {
            ch = -ch;
            cl = -cl;
          }
          T xv[VEC];
          R.fetch(w, int(iq[h]), col, cvalid, xv);
#pragma unroll
          for (int u = 0; u < VEC; ++u) acc[u].fma(ch, cl, xv[u]);
        }
        if (cnt == 255) {
          // hits beyond the list: found again, in the same order
          Cursor cur;
          cur.start(m, hp.n_hg, H.mask, H.shift);
          int nh = 0;
          while (cur.valid()) {
            int i1, s1, g1;
            cur.take(i1, s1, g1, H.mask, H.shift);
            const int q = lookup<MODE>(w, m ^ ((1u | (1u << s1)) << i1));
            if (q < 0) continue;
            if (nh++ < kHitCap) continue;
            T ch = coef_hi<T>(H.hi, H.t, g1), cl = coef_lo<T>(H.lo, g1);
            if (__popc(m & between_bits(i1, s1)) & 1) {
              ch = -ch;
              cl = -cl;
            }
            T xv[VEC];
            R.fetch(w, q, col, cvalid, xv);
#pragma unroll
            for (int u = 0; u < VEC; ++u) acc[u].fma(ch, cl, xv[u]);
          }
        }
        T out[VEC];
        if (PASS_A) {
          T xv[VEC], yv[VEC];
          C::load(x + int64_t(k) * ld + col, cvalid, xv);
          C::load(y + int64_t(k) * ld + col, cvalid, yv);
          const Coef<T> dc = diag_of<T>(hp, H.dhi, H.dlo, H.d64, __ldg(L.blk_major + b), m);
#pragma unroll
          for (int u = 0; u < VEC; ++u) {
            acc[u].fma(dc.hi, dc.lo, xv[u]);
            out[u] = acc[u].value() + yv[u];
          }
        } else {
#pragma unroll
          for (int u = 0; u < VEC; ++u) out[u] = acc[u].value();
        }
        C::store(y + orow * ld + col, cvalid, out);
      }
    }
    __syncthreads();
  }
}

template <typename T, int VEC, int G, bool PASS_A>
__global__ void __launch_bounds__(kHThreads) hv_hashm_kernel(const HvArgs a, const HamParams hp) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ HopSmem H;
  __shared__ uint32_t lq[kHThreads * kHitCap];
  __shared__ uint8_t lg[kHThreads * kHitCap];
  __shared__ uint8_t lcnt[kHThreads];
  const ItemSmem sm = item_smem_of(a, s_dyn);
  load_hops(hp, H);
  for (int ii = blockIdx.x; ii < a.n_hitems; ii += gridDim.x) {
    const HItem it = a.items[ii];
    __syncthreads();
    const int mode = item_mode(a, it, sm);
    if (mode == 0) {
      build_item<T, PASS_A, false>(a, it, sm, static_cast<T*>(nullptr));
      multi_item<T, VEC, G, PASS_A, 0>(a, hp, it, sm, H, lq, lg, lcnt);
    } else if (mode == 1) {
      multi_item<T, VEC, G, PASS_A, 1>(a, hp, it, sm, H, lq, lg, lcnt);
    } else {
      multi_item<T, VEC, G, PASS_A, 2>(a, hp, it, sm, H, lq, lg, lcnt);
    }
  }
}

int ceil_log2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

// Items and block tables of one layout for item size hcap.
cudaError_t build_hash(mcd_ctx* c, Layout& L, int hcap) {
  cudaStream_t s = c->stream;
  std::vector<uint32_t> off(size_t(L.nblk) + 1);
  cudaError_t e = cudaMemcpyAsync(off.data(), L.blk_off, off.size() * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  std::vector<HItem> items;
  std::vector<uint32_t> big;   // item index of the first chunk of each tabled block
  int64_t tab_len = 0, flt_len = 0;
  int64_t b0 = 0;
  auto flush = [&](int64_t b1) {
    if (b1 > b0) items.push_back(HItem{off[b0], off[b1], uint32_t(b0), uint32_t(b1), 0u, 0u, 0u, 0u});
    b0 = b1;
  };
  for (int64_t b = 0; b < L.nblk; ++b) {
    const int64_t K = int64_t(off[b + 1]) - off[b];
    if (K > hcap) {
      flush(b);
      uint32_t lg = kHashSearch, toff = 0, lf = 0, foff = 0;
      if (K <= kMaxBlockTable) {
        lg = uint32_t(ceil_log2(2 * K));
        toff = uint32_t(tab_len);
        tab_len += int64_t(1) << lg;
        lf = uint32_t(ceil_log2(16 * K));
        foff = uint32_t(flt_len);
        flt_len += (int64_t(1) << lf) / 32;
        big.push_back(uint32_t(items.size()));
      }
      for (int64_t c0 = off[b]; c0 < off[b + 1]; c0 += hcap)
        items.push_back(HItem{uint32_t(c0), uint32_t(std::min<int64_t>(c0 + hcap, off[b + 1])), uint32_t(b),
                              uint32_t(b + 1), toff, lg, foff, lf});
      b0 = b + 1;
    } else if (int64_t(off[b + 1]) - off[b0] > hcap) {
      flush(b);
    }
  }
  flush(L.nblk);
  if (tab_len > 0xFFFFFFFFll || flt_len > 0xFFFFFFFFll) return cudaErrorInvalidValue;
  if (int64_t(items.size()) > L.hitem_cap) {
    if (L.hitems) cudaFreeAsync(L.hitems, c->stream);
    L.hitems = nullptr;
    L.hitem_cap = 0;
    e = cudaMallocAsync(&L.hitems, items.size() * sizeof(HItem), c->stream);
    if (e != cudaSuccess) return e;
    L.hitem_cap = int64_t(items.size());
  }
  if (tab_len > L.htab_cap) {
    if (L.htab) cudaFreeAsync(L.htab, c->stream);
    L.htab = nullptr;
    L.htab_cap = 0;
    e = cudaMallocAsync(&L.htab, size_t(tab_len) * 4, c->stream);
    if (e != cudaSuccess) return e;
    L.htab_cap = tab_len;
  }
  if (flt_len > L.hflt_cap) {
    if (L.hflt) cudaFreeAsync(L.hflt, c->stream);
    L.hflt = nullptr;
    L.hflt_cap = 0;
    e = cudaMallocAsync(&L.hflt, size_t(flt_len) * 4, c->stream);
    if (e != cudaSuccess) return e;
    L.hflt_cap = flt_len;
  }
  L.n_hitems = int64_t(items.size());
  L.htab_len = tab_len;
  L.hflt_len = flt_len;
  e = cudaMemcpyAsync(L.hitems, items.data(), items.size() * sizeof(HItem), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && tab_len > 0) e = cudaMemsetAsync(L.htab, 0xFF, size_t(tab_len) * 4, s);
  if (e == cudaSuccess && flt_len > 0) e = cudaMemsetAsync(L.hflt, 0, size_t(flt_len) * 4, s);
  uint32_t* d_big = nullptr;
  if (e == cudaSuccess && !big.empty()) {
    e = cudaMallocAsync(&d_big, big.size() * 4, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_big, big.data(), big.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      block_tables_kernel<<<int(big.size()), 256, 0, s>>>(L, d_big, int(big.size()), L.htab, L.hflt, L.hitems);
      MCD_LAUNCHED(c);
      e = cudaGetLastError();
    }
    cudaFreeAsync(d_big, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host vectors die here
  if (e == cudaSuccess) L.hash_built = hcap;
  return e;
}

// shared memory of an item: table (4 * hcap slots), words, block offsets and
// indices, then (single column) the staged x
size_t item_base_bytes(const HvArgs& a) {
  const size_t off = (size_t(1) << a.hlog2) * 4 + (size_t(1) << a.flog2) / 8 + size_t(a.hcap) * 4 +
                     (size_t(a.hcap) * 2 + 2) * 2;
  return (off + 15) & ~size_t(15);
}

size_t item_smem(const HvArgs& a, size_t xs_elem) { return item_base_bytes(a) + size_t(a.hcap) * xs_elem; }

HvArgs hash_args(mcd_ctx* c, const void* x, void* y, int ncols, int ld) {
  HvArgs a{};
  a.x = x;
  a.y = y;
  a.ncols = ncols;
  a.ld = ld;
  a.n_sites = c->n;
  a.hcap = c->hash_item;
  a.hlog2 = ceil_log2(4 * int64_t(c->hash_item));
  a.flog2 = ceil_log2(32 * int64_t(c->hash_item));
  a.off_xs = int(item_base_bytes(a));
  return a;
}

template <typename T>
cudaError_t launch_hash1(mcd_ctx* c, const void* x, void* y, int ld, double* partials, int max_parts,
                         unsigned int* ticket, double* dot_out) {
  HvArgs a = hash_args(c, x, y, 1, ld);
  a.dot_partials = partials;
  a.ticket = ticket;
  a.dot_out = dot_out;
  const size_t smem = item_smem(a, sizeof(T));
  static std::atomic<int> configured{-1};
  if (configured < int(smem)) {
    cudaFuncSetAttribute(hv_hash1_kernel<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(hv_hash1_kernel<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(hv_hash1_kernel<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    configured = int(smem);
  }
  const int cap = device_sms() * 32;
  for (int pass = 0; pass < 2; ++pass) {
    const Layout& L = pass ? c->idx.A : c->idx.B;
    a.L = L;
    a.items = L.hitems;
    a.n_hitems = int(L.n_hitems);
    a.htab = L.htab;
    a.hflt = L.hflt;
    int grid = int(std::min<int64_t>(L.n_hitems, cap));
    if (grid < 1) grid = 1;
    timing_begin(c, pass);
    if (pass == 0) {
      hv_hash1_kernel<T, false, false><<<grid, kHThreads, smem, c->stream>>>(a, *c->hp);
    } else if (partials) {
      grid = std::min(grid, max_parts);
      hv_hash1_kernel<T, true, true><<<grid, kHThreads, smem, c->stream>>>(a, *c->hp);
    } else {
      hv_hash1_kernel<T, true, false><<<grid, kHThreads, smem, c->stream>>>(a, *c->hp);
    }
    MCD_LAUNCHED(c);
    timing_end(c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T, int VEC, int G>
cudaError_t launch_hashm(mcd_ctx* c, const void* x, void* y, int ncols, int ld) {
  HvArgs a = hash_args(c, x, y, ncols, ld);
  const size_t smem = item_smem(a, 0);
  static std::atomic<int> configured{-1};
  if (configured < int(smem)) {
    cudaFuncSetAttribute(hv_hashm_kernel<T, VEC, G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(hv_hashm_kernel<T, VEC, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    configured = int(smem);
  }
  const int cap = device_sms() * 32;
  for (int pass = 0; pass < 2; ++pass) {
    const Layout& L = pass ? c->idx.A : c->idx.B;
    a.L = L;
    a.items = L.hitems;
    a.n_hitems = int(L.n_hitems);
    a.htab = L.htab;
    a.hflt = L.hflt;
    int grid = int(std::min<int64_t>(L.n_hitems, cap));
    if (grid < 1) grid = 1;
    timing_begin(c, pass);
    if (pass == 0)
      hv_hashm_kernel<T, VEC, G, false><<<grid, kHThreads, smem, c->stream>>>(a, *c->hp);
    else
      hv_hashm_kernel<T, VEC, G, true><<<grid, kHThreads, smem, c->stream>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T, int VEC>
cudaError_t dispatch_hashm(mcd_ctx* c, const void* x, void* y, int ncols, int ld) {
  const int chunks = (ncols + VEC - 1) / VEC;
  if (chunks <= 1) return launch_hashm<T, VEC, 1>(c, x, y, ncols, ld);
  if (chunks <= 2) return launch_hashm<T, VEC, 2>(c, x, y, ncols, ld);
  if (chunks <= 4) return launch_hashm<T, VEC, 4>(c, x, y, ncols, ld);
  if (chunks <= 8) return launch_hashm<T, VEC, 8>(c, x, y, ncols, ld);
  return launch_hashm<T, VEC, 16>(c, x, y, ncols, ld);
}

}  // namespace

bool hash_eligible(const mcd_ctx* c) {
  return c->hp->n_hg > 0 && (c->hv_algo == 3 || (c->hv_algo == 0 && c->n > 16));
}

void free_hash(Layout& L, cudaStream_t s) {
  if (L.hitems) cudaFreeAsync(L.hitems, s);
  if (L.htab) cudaFreeAsync(L.htab, s);
  if (L.hflt) cudaFreeAsync(L.hflt, s);
  L.hitems = nullptr;
  L.htab = nullptr;
  L.hflt = nullptr;
  L.hitem_cap = L.htab_cap = L.hflt_cap = 0;
  L.n_hitems = L.htab_len = L.hflt_len = 0;
  L.hash_built = 0;
}

int hash_apply(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, double* dot_partials,
               int max_parts, unsigned int* ticket, double* dot_out) {
  for (Layout* L : {&c->idx.B, &c->idx.A}) {
    if (L->hash_built == c->hash_item) continue;
    const cudaError_t e = build_hash(c, *L, c->hash_item);
    if (e != cudaSuccess) return cuda_fail(c, e, "hash index");
  }
  const bool vec_ok = ncols > 1 && ld % (dtype == MCD_F64 ? 2 : 4) == 0 &&
                      reinterpret_cast<uintptr_t>(x) % 16 == 0 && reinterpret_cast<uintptr_t>(y) % 16 == 0;
  cudaError_t e;
  if (dtype == MCD_F64) {
    if (ncols == 1) e = launch_hash1<double>(c, x, y, ld, dot_partials, max_parts, ticket, dot_out);
    else if (vec_ok) e = dispatch_hashm<double, 2>(c, x, y, ncols, ld);
    else e = dispatch_hashm<double, 1>(c, x, y, ncols, ld);
  } else {
    if (ncols == 1) e = launch_hash1<float>(c, x, y, ld, dot_partials, max_parts, ticket, dot_out);
    else if (vec_ok) e = dispatch_hashm<float, 4>(c, x, y, ncols, ld);
    else e = dispatch_hashm<float, 1>(c, x, y, ncols, ld);
  }
  return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "hash H*v launch");
}

}  // namespace mcd
