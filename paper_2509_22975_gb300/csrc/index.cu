// Device index of a truncated basis (built once per basis).
//
// The basis F~ is a sorted array of words w = (up << n) | dn (Sec. "Subspace of
// the ground state" keeps F~ as a searchable set; sorting replaces the
// paper's binary tree).  Sorting by word groups states that share an up word
// into contiguous blocks, so a down-spin hop (which keeps the up word) lands
// in the same block.  A second, dn-major ordering groups states that share a
// down word, so an up-spin hop stays inside a block of that ordering.  For
// each ordering this file builds:
//   minor[k]      the half of the word that hops move (dn in A, up in B),
//   blk_off[b]    first position of block b (blk_off[nblk] = n),
//   blk_major[b]  the half shared by block b,
//   item_blk[i]   block containing position i * kItem (work-item start),
// and for B the permutation perm[k] = basis index of dn-major position k,
// obtained by a stable LSD radix sort of the dn words (stable, so equal dn
// words keep ascending up order).
#include "mcd_internal.h"

namespace mcd {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048
constexpr int kRadixBits = 8;
constexpr int kRadixDigits = 1 << kRadixBits;

// ---- exclusive scan of uint32 (tile sums, recursive) ----------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void scan_tiles_kernel(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tile_sums) {
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

__global__ void add_tile_offsets_kernel(uint32_t* out, int64_t n, const uint32_t* offs) {
  const int64_t base = int64_t(blockIdx.x) * kScanTile;
  const uint32_t o = offs[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
    if (base + k < n) out[base + k] += o;
}

// ---- radix sort (stable, 8-bit digits) -------------------------------------------------
__global__ void radix_hist_kernel(const uint32_t* keys, int64_t n, int shift, uint32_t* hist,
                                  int64_t ntiles) {
  __shared__ uint32_t h[kRadixDigits];
  for (int d = threadIdx.x; d < kRadixDigits; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
    if (base + k < n) atomicAdd(&h[(keys[base + k] >> shift) & (kRadixDigits - 1)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadixDigits; d += blockDim.x) hist[int64_t(d) * ntiles + blockIdx.x] = h[d];
}

// Each tile is handled in kScanItems rounds of kScanThreads consecutive keys;
// within a round a key's rank among equal digits comes from the lower lanes
// of its warp (match) and the lower warps (shared counts), so the scatter
// keeps input order (stable).
__global__ void radix_scatter_kernel(const uint32_t* keys_in, const uint32_t* vals_in, int64_t n,
                                     int shift, const uint32_t* offs, int64_t ntiles,
                                     uint32_t* keys_out, uint32_t* vals_out) {
  constexpr int kWarps = kScanThreads / 32;
  __shared__ uint32_t run[kRadixDigits];
  __shared__ uint32_t wc[kWarps][kRadixDigits];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadixDigits; d += blockDim.x) run[d] = offs[int64_t(d) * ntiles + blockIdx.x];
  const int64_t base = int64_t(blockIdx.x) * kScanTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kScanItems; ++r) {
    for (int k = threadIdx.x; k < kWarps * kRadixDigits; k += blockDim.x) (&wc[0][0])[k] = 0;
    __syncthreads();
    const int64_t i = base + int64_t(r) * kScanThreads + threadIdx.x;
    const bool ok = i < n;
    uint32_t key = ok ? keys_in[i] : 0u;
    const int d = ok ? int((key >> shift) & (kRadixDigits - 1)) : kRadixDigits;   // kRadixDigits = none
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (ok && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      uint32_t pos = run[d] + rank;
      for (int w = 0; w < warp; ++w) pos += wc[w][d];
      keys_out[pos] = key;
      vals_out[pos] = vals_in ? vals_in[i] : uint32_t(i);
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kRadixDigits; dd += blockDim.x) {
      uint32_t s = 0;
      for (int w = 0; w < kWarps; ++w) s += wc[w][dd];
      run[dd] += s;
    }
    __syncthreads();
  }
}

// ---- layouts --------------------------------------------------------------------------
__global__ void split_words_kernel(const uint64_t* words, int64_t n, int nsites, uint32_t* dn,
                                   uint32_t* up) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint64_t w = words[k];
  dn[k] = uint32_t(nsites == 32 ? (w & 0xFFFFFFFFull) : (w & ((1ull << nsites) - 1)));
  up[k] = uint32_t(w >> nsites);
}

__global__ void gather_u32_kernel(const uint32_t* src, const uint32_t* perm, int64_t n, uint32_t* dst) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < n) dst[k] = src[perm[k]];
}

// flag[k] = 1 at the first position of each block of equal `major`
__global__ void block_flags_kernel(const uint32_t* major, int64_t n, uint32_t* flag) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < n) flag[k] = (k == 0 || major[k] != major[k - 1]) ? 1u : 0u;
}

// scan = exclusive scan of flags: block id of k = scan[k] + flag[k] - 1
__global__ void block_tables_kernel(const uint32_t* major, const uint32_t* flag, const uint32_t* scan,
                                    int64_t n, uint32_t* blk_off, uint32_t* blk_major,
                                    uint32_t* item_blk) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t b = scan[k] + flag[k] - 1u;
  if (flag[k]) {
    blk_off[b] = uint32_t(k);
    blk_major[b] = major[k];
  }
  if (k % kItem == 0) item_blk[k / kItem] = b;
  if (k == n - 1) {
    blk_off[b + 1] = uint32_t(n);
    item_blk[(n + kItem - 1) / kItem] = b + 1;   // sentinel: nblk
  }
}

// ---- checks --------------------------------------------------------------------------
// bit 0: not strictly ascending; bit 1: word outside the (n_up, n_dn) sector
__global__ void check_basis_kernel(const uint64_t* w, int64_t n, int nsites, int n_up, int n_dn,
                                   unsigned int* bad) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint64_t x = w[k];
  if (k > 0 && x <= w[k - 1]) atomicOr(bad, 1u);
  const uint64_t half = nsites == 32 ? 0xFFFFFFFFull : ((1ull << nsites) - 1);
  const bool high = nsites < 32 && (x >> (2 * nsites)) != 0;
  if (high || __popcll(x >> nsites) != n_up || __popcll(x & half) != n_dn) atomicOr(bad, 2u);
}

struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~DevBuf() { if (p) cudaFreeAsync(p, s); }
};

int grid_of(int64_t n, int t) { return int((n + t - 1) / t); }

}  // namespace

// exclusive scan of n uint32 values (in may equal out)
cudaError_t scan_u32(mcd_ctx* c, const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (ntiles == 1) {
    scan_tiles_kernel<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    MCD_LAUNCHED(c);
    return cudaGetLastError();
  }
  uint32_t* sums = nullptr;
  cudaError_t e = cudaMallocAsync(&sums, ntiles * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  scan_tiles_kernel<<<int(ntiles), kScanThreads, 0, s>>>(in, out, n, sums);
  MCD_LAUNCHED(c);
  e = scan_u32(c, sums, sums, ntiles, s);
  if (e == cudaSuccess) {
    add_tile_offsets_kernel<<<int(ntiles), kScanThreads, 0, s>>>(out, n, sums);
    MCD_LAUNCHED(c);
    e = cudaGetLastError();
  }
  cudaFreeAsync(sums, s);
  return e;
}

// Build blocks of equal `major` over an ordering of n states.
static cudaError_t build_layout(mcd_ctx* c, const uint32_t* major, int64_t n, Layout& L, uint32_t* tmp_flag,
                                uint32_t* tmp_scan, cudaStream_t s) {
  const int T = 256;
  block_flags_kernel<<<grid_of(n, T), T, 0, s>>>(major, n, tmp_flag);
  MCD_LAUNCHED(c);
  cudaError_t e = scan_u32(c, tmp_flag, tmp_scan, n, s);
  if (e != cudaSuccess) return e;
  uint32_t last_scan = 0, last_flag = 0;
  e = cudaMemcpyAsync(&last_scan, tmp_scan + n - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&last_flag, tmp_flag + n - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  L.n = n;
  L.nblk = int64_t(last_scan) + last_flag;
  L.n_items = (n + kItem - 1) / kItem;
  L.hash_built = 0;   // hash items describe the previous basis
  cache_invalidate(L);
  block_tables_kernel<<<grid_of(n, T), T, 0, s>>>(major, tmp_flag, tmp_scan, n, L.blk_off,
                                                  L.blk_major, L.item_blk);
  MCD_LAUNCHED(c);
  return cudaGetLastError();
}

void free_index(DevIndex& ix, cudaStream_t s) {
  auto f = [s](void* p) { if (p) cudaFreeAsync(p, s); };
  f(ix.words);
  for (Layout* L : {&ix.A, &ix.B}) {
    f(L->minor); f(L->blk_off); f(L->blk_major); f(L->item_blk); f(L->perm);
    free_hash(*L, s);
    free_cache(*L, s);
    *L = Layout();
  }
  ix.words = nullptr;
  ix.n = 0;
  ix.cap = 0;
  ix.nnz = -1;
}

// Persistent index buffers sized for `cap` states; kept across bases that fit.
static cudaError_t reserve_index(DevIndex& ix, int64_t n, cudaStream_t s) {
  if (ix.cap >= n && ix.words) return cudaSuccess;
  free_index(ix, s);
  const int64_t items = (n + kItem - 1) / kItem + 1;
  // words and perm end 16 bytes past the last state: the streaming H~v kernel
  // copies aligned 16-byte units that cover a range of states
  cudaError_t e = cudaMallocAsync(&ix.words, (n + 2) * sizeof(uint64_t), s);
  for (Layout* L : {&ix.A, &ix.B}) {
    if (e == cudaSuccess) e = cudaMallocAsync(&L->minor, n * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&L->blk_off, (n + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&L->blk_major, n * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&L->item_blk, items * 4, s);
  }
  if (e == cudaSuccess) e = cudaMallocAsync(&ix.B.perm, (n + 4) * 4, s);
  if (e != cudaSuccess) {
    free_index(ix, s);
    return e;
  }
  ix.cap = n;
  return cudaSuccess;
}

int build_index(mcd_ctx* c, const uint64_t* words, int64_t n, bool on_device) {
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  DevIndex& ix = c->idx;
  cudaStream_t s = c->stream;
  const int T = 256;
  e = reserve_index(ix, n, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(index)");
  ix.n = n;
  ix.nnz = -1;
  e = cudaMemcpyAsync(ix.words, words, n * sizeof(uint64_t),
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    free_index(ix, s);
    return cuda_fail(c, e, "copy words");
  }
  {
    unsigned int* bad = nullptr;
    unsigned int hbad = 0;
    e = cudaMallocAsync(&bad, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, 4, s);
    if (e == cudaSuccess) {
      check_basis_kernel<<<grid_of(n, T), T, 0, s>>>(ix.words, n, c->n, c->n_up, c->n_dn, bad);
      MCD_LAUNCHED(c);
      e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(bad, s);
    if (e != cudaSuccess) {
      free_index(ix, s);
      return cuda_fail(c, e, "basis check");
    }
    if (hbad & 1u) {
      free_index(ix, s);
      return fail(c, MCD_E_INVALID, "basis words must be strictly ascending");
    }
    if (hbad & 2u) {
      free_index(ix, s);
      return fail(c, MCD_E_SECTOR, "word outside the (N_up, N_dn) sector");
    }
  }
  // halves
  uint32_t *up = nullptr, *flag = nullptr, *scn = nullptr, *k2 = nullptr, *v2 = nullptr, *hist = nullptr;
  e = cudaMallocAsync(&up, n * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&flag, n * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&scn, n * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&k2, n * 4, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&v2, n * 4, s);
  const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (e == cudaSuccess) e = cudaMallocAsync(&hist, ntiles * kRadixDigits * 4, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(up, s); cudaFreeAsync(flag, s); cudaFreeAsync(scn, s);
    cudaFreeAsync(k2, s); cudaFreeAsync(v2, s); cudaFreeAsync(hist, s);
    return cuda_fail(c, e, "cudaMalloc(index)");
  }
  split_words_kernel<<<grid_of(n, T), T, 0, s>>>(ix.words, n, c->n, ix.A.minor, up);
  MCD_LAUNCHED(c);
  e = build_layout(c, up, n, ix.A, flag, scn, s);
  // dn-major: stable sort of the dn words with values = basis index.
  // ping-pong between (keys_a = scn, vals_a = B.perm) and (k2, v2)
  if (e == cudaSuccess) {
    const int passes = (c->n + kRadixBits - 1) / kRadixBits;
    const uint32_t* kin = ix.A.minor;
    const uint32_t* vin = nullptr;   // identity
    uint32_t* bufk[2] = {scn, k2};
    uint32_t* bufv[2] = {ix.B.perm, v2};
    // make the last pass land in (scn, B.perm)
    int which = (passes % 2 == 1) ? 0 : 1;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
      const int shift = p * kRadixBits;
      radix_hist_kernel<<<int(ntiles), kScanThreads, 0, s>>>(kin, n, shift, hist, ntiles);
      MCD_LAUNCHED(c);
      e = scan_u32(c, hist, hist, ntiles * kRadixDigits, s);
      if (e != cudaSuccess) break;
      radix_scatter_kernel<<<int(ntiles), kScanThreads, 0, s>>>(kin, vin, n, shift, hist, ntiles,
                                                                bufk[which], bufv[which]);
      MCD_LAUNCHED(c);
      e = cudaGetLastError();
      kin = bufk[which];
      vin = bufv[which];
      which ^= 1;
    }
    // keys (dn words, dn-major) now in scn, perm in B.perm
    if (e == cudaSuccess) {
      gather_u32_kernel<<<grid_of(n, T), T, 0, s>>>(up, ix.B.perm, n, ix.B.minor);
      MCD_LAUNCHED(c);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      // scn holds dn-major dn words; blocks of equal dn.  flag/up reused as temps.
      e = cudaMemcpyAsync(k2, scn, n * 4, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = build_layout(c, k2, n, ix.B, flag, scn, s);
    }
  }
  cudaFreeAsync(up, s); cudaFreeAsync(flag, s); cudaFreeAsync(scn, s);
  cudaFreeAsync(k2, s); cudaFreeAsync(v2, s); cudaFreeAsync(hist, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_index(ix, s);
    return cuda_fail(c, e, "index build");
  }
  return MCD_OK;
}

}  // namespace mcd
