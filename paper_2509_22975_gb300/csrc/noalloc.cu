// mcd_connections_noalloc: the connection-list dump of mcd_connections for
// callers that must not allocate device memory.
//
// mcd_connections needs per-row counts and offsets and takes them from the
// stream-ordered allocator on every call.  Some callers cannot allow that:
// an application that hands all device memory to its own pool at start-up
// and forbids any later allocation by a library, or a caller that runs under
// a fixed memory budget where a late allocation can fail.  This variant keeps
// its scratch in one fixed array in device global memory instead:
//
//   g_noalloc_scratch: kNoAllocMaxStates per-row counts, kNoAllocMaxStates
//   per-row offsets (reused as write cursors) and the total, 2 MiB in all.
//   Every GPU that loads the library holds this array until the process
//   exits.  Bases above kNoAllocMaxStates states are rejected.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and keeps it for the life of the process; that first
// call should come before any stream capture.  The kept address belongs to
// the device's primary context: after the application resets the device
// (cudaDeviceReset), calls of this entry point are not supported.  Every call
// reuses the same array and leaves its contents behind: the counts are
// cleared at the start of each call, and calls whose work overlaps on the GPU
// (two streams, or two contexts on one device) race on it.
#include <mutex>

#include "mcd_internal.h"

namespace mcd {
namespace {

constexpr int64_t kNoAllocMaxStates = int64_t(1) << 18;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;

static __device__ __align__(256) uint32_t g_noalloc_scratch[2 * kNoAllocMaxStates + 4];

std::mutex g_setup_mutex;
uint32_t* g_scratch_addr[kMaxDevices] = {};

// Address of g_noalloc_scratch on `device` (which must be current).
int scratch_address(mcd_ctx* c, uint32_t** out) {
  if (c->device < 0 || c->device >= kMaxDevices) return fail(c, MCD_E_INVALID, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[c->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_addr[c->device] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_addr[c->device];
  return MCD_OK;
}

__device__ __forceinline__ int na_find(const uint32_t* a, int lo, int hi, uint32_t key) {
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

// One thread per state of a layout: count (write == 0) or emit its in-basis
// hop targets.  Counts go to cnt[row] by atomic add; entries go to the slots
// reserved by atomic increments of cursor[row].
template <bool PASS_A>
__global__ void na_conn_kernel(const Layout L, const HamParams hp, uint32_t* cnt, uint32_t* cursor,
                               int64_t* rows, int64_t* cols, double* vals, int write) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= L.n) return;
  int64_t lo = 0, len = L.nblk;
  while (len > 1) {
    const int64_t h = len >> 1;
    if (L.blk_off[lo + h] <= uint32_t(k)) lo += h;
    len -= h;
  }
  const int bbase = int(L.blk_off[lo]), bend = int(L.blk_off[lo + 1]);
  const uint32_t m = L.minor[k];
  const int64_t row = PASS_A ? k : int64_t(L.perm[k]);
  uint32_t found = 0;
  for (int b = 0; b < hp.n_bonds; ++b) {
    const uint32_t mk = hp.bonds[b].mask;
    if (__popc(m & mk) != 1) continue;
    const int q = na_find(L.minor, bbase, bend, m ^ mk);
    if (q < 0) continue;
    if (write) {
      const uint32_t pos = atomicAdd(&cursor[row], 1u);
      rows[pos] = row;
      cols[pos] = PASS_A ? int64_t(q) : int64_t(L.perm[q]);
      vals[pos] = (__popc(m & hp.bonds[b].between) & 1) ? -hp.bonds[b].t : hp.bonds[b].t;
    }
    ++found;
  }
  if (!write && found) atomicAdd(&cnt[row], found);
}

// off = exclusive scan of cnt[0, n), *total = sum; one block (n <= 2^18).
__global__ void na_scan_kernel(const uint32_t* cnt, uint32_t* off, int64_t n, uint32_t* total) {
  __shared__ uint32_t s[kScanThreads];
  const int t = threadIdx.x;
  const int64_t chunk = (n + kScanThreads - 1) / kScanThreads;
  const int64_t lo = t * chunk, hi = (lo + chunk < n) ? lo + chunk : n;
  uint32_t sum = 0;
  for (int64_t i = lo; i < hi; ++i) sum += cnt[i];
  s[t] = sum;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {
    const uint32_t v = t >= o ? s[t - o] : 0u;
    __syncthreads();
    s[t] += v;
    __syncthreads();
  }
  uint32_t run = s[t] - sum;
  for (int64_t i = lo; i < hi; ++i) {
    off[i] = run;
    run += cnt[i];
  }
  if (t == kScanThreads - 1) *total = s[t];
}

int grid_of(int64_t n, int t) { return int((n + t - 1) / t); }

}  // namespace
}  // namespace mcd

using namespace mcd;

extern "C" int mcd_connections_noalloc(mcd_ctx* c, int64_t* rows, int64_t* cols, double* vals, int64_t cap,
                                       int64_t* nnz) {
  if (!c || !nnz) return MCD_E_INVALID;
  if (!c->has_ham || c->n_basis == 0) return fail(c, MCD_E_STATE, "no Hamiltonian or basis set");
  if (c->device < 0) return fail(c, MCD_E_NODEVICE, "host-only context (device = -1)");
  if (rows && (!cols || !vals)) return fail(c, MCD_E_INVALID, "rows, cols and vals go together");
  const int64_t n = c->idx.n;
  if (n > kNoAllocMaxStates)
    return fail(c, MCD_E_INVALID,
                "basis has " + std::to_string(n) + " states; mcd_connections_noalloc handles at most " +
                    std::to_string(kNoAllocMaxStates) + " (its fixed scratch size)");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  uint32_t* base = nullptr;
  int st = scratch_address(c, &base);
  if (st != MCD_OK) return st;
  uint32_t* cnt = base;
  uint32_t* off = base + kNoAllocMaxStates;
  uint32_t* tot = base + 2 * kNoAllocMaxStates;
  cudaStream_t s = c->stream;
  e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * size_t(n), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "clear no-alloc scratch");
  na_conn_kernel<false><<<grid_of(n, kThreads), kThreads, 0, s>>>(c->idx.B, *c->hp, cnt, nullptr, nullptr,
                                                                   nullptr, nullptr, 0);
  MCD_LAUNCHED(c);
  na_conn_kernel<true><<<grid_of(n, kThreads), kThreads, 0, s>>>(c->idx.A, *c->hp, cnt, nullptr, nullptr,
                                                                  nullptr, nullptr, 0);
  MCD_LAUNCHED(c);
  na_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, off, n, tot);
  MCD_LAUNCHED(c);
  uint32_t total = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "no-alloc connection count");
  *nnz = int64_t(total);
  c->idx.nnz = int64_t(total);
  if (!rows) return MCD_OK;
  if (int64_t(total) > cap) return fail(c, MCD_E_INVALID, "connections: capacity too small");
  na_conn_kernel<false><<<grid_of(n, kThreads), kThreads, 0, s>>>(c->idx.B, *c->hp, nullptr, off, rows, cols,
                                                                   vals, 1);
  MCD_LAUNCHED(c);
  na_conn_kernel<true><<<grid_of(n, kThreads), kThreads, 0, s>>>(c->idx.A, *c->hp, nullptr, off, rows, cols,
                                                                  vals, 1);
  MCD_LAUNCHED(c);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? MCD_OK : cuda_fail(c, e, "no-alloc connection write");
}
