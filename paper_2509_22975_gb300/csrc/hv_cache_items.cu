// Connection-cache H~V for many columns, CTA per work item: the x rows of
// the item's stage range are staged in shared memory with ordinary loads
// when they fit (48 KiB), else gathered from global memory (L2); groups of G
// lanes share a state, lane g owning VEC columns.  Pass B (up-spin hops,
// dn-major blocks) reads a dn-major copy of X made by permute_rows_kernel,
// so that the rows of its blocks are contiguous.  Many CTAs per SM hide the
// latency of the unstaged gathers: the better kernel where most states sit
// in blocks far larger than a work item (the 6x4 cluster); the pipelined
// tiles of hv_cache_cols.cu are better where blocks can be staged.  The
// first many-column product of a width times both and keeps the faster
// (MCD_OPT_HV_COLS).  The records and their layout are those of hv_cache.cu.
#include <atomic>
#include <algorithm>

#include "hv_cache.cuh"

namespace mcd {
namespace {

// Many columns (or one column with a row stride): CTA per item, x rows of the
// stage range staged with ordinary loads when they fit, G lanes per state.
template <typename T, int VEC, int G, bool PASS_A>
__global__ void __launch_bounds__(kCT) hv_item_kernel(const CArgs a, const HamParams hp) {
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
  using C = ChunkOf<T, VEC>;
  constexpr int kSPW = 32 / G;                   // states of a slice processed at once by a warp
  constexpr int kU = VEC == 1 ? 8 : 4;           // record groups in flight per lane
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane % G, tg = lane / G;
  const bool lane_ok = tg < kSPW;                // G not dividing 32 leaves lanes idle
  const int col0 = g * VEC;
  const int cvalid = a.ncols - col0;
  const T* __restrict__ x = static_cast<const T*>(a.x);
  T* __restrict__ y = static_cast<T*>(a.y);
  const unsigned char* recg = static_cast<const unsigned char*>(a.rec);
  const uint32_t half = a.n_sites >= 32 ? 0xFFFFFFFFu : ((1u << a.n_sites) - 1u);
  const int ld = a.ld, ncp = a.ncp;
  const int ldx = a.x_layout ? ncp : ld;   // row stride of x (pass B may read the dn-major copy)

  for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
    const CItem it = a.items[item];
    const uint32_t sb = a.blk_off[it.b0], se = a.blk_off[it.b1 + 1];
    const int nst = int(se - sb);
    const bool staged = int64_t(nst) * ncp <= a.xs_cap;
    __syncthreads();   // the previous item's rows are no longer read
    if (staged && lane_ok && cvalid > 0) {
      for (int q = warp * kSPW + tg; q < nst; q += kCWarps * kSPW) {
        const int64_t row = (PASS_A || a.x_layout) ? int64_t(sb) + q : int64_t(__ldg(a.perm + sb + q));
        T v[VEC];
        C::load(x + row * ldx + col0, cvalid, v);
#pragma unroll
        for (int u = 0; u < VEC; ++u) xs[q * ncp + col0 + u] = v[u];
      }
    }
    __syncthreads();
    const bool wide = (it.flags & 1u) != 0u;
    auto gather = [&](int q, T* v) {
      if (staged) {
#pragma unroll
        for (int u = 0; u < VEC; ++u) v[u] = xs[q * ncp + col0 + u];
      } else {
        const int64_t row = (PASS_A || a.x_layout) ? int64_t(sb) + q : int64_t(__ldg(a.perm + sb + q));
        C::load(x + row * ldx + col0, cvalid, v);
      }
    };
    const int nsl = int((it.hi - it.lo + 31) / 32);
    for (int pass = 0;; ++pass) {   // serpentine slice order (see serp_slice)
      const int sl = serp_slice(pass, warp, kCWarps);
      if (sl >= nsl) break;
      const int64_t s = int64_t(it.slice0) + sl;
      const uint32_t ga = __ldg(a.col + s), gz = __ldg(a.col + s + 1);
      const uint32_t locs = __ldg(a.smap + s * 32 + lane);   // the slice's lane map, one load per warp
      for (int t0 = 0; t0 < 32; t0 += kSPW) {
        const int t = t0 + tg;
        const uint16_t loc = uint16_t(__shfl_sync(0xffffffffu, locs, t & 31));
        if (!lane_ok || cvalid <= 0 || t >= 32) continue;   // idle lanes: past the last column chunk
        if (loc == kNoState) continue;                      // empty lanes are the slice's last ones
        const uint32_t k = it.lo + loc;
        const unsigned char* rp = recg + int64_t(ga) * kGroup + t * kLaneBytes;
        Acc<T> acc[VEC];
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[u].zero();
        if (wide)
          state_sum<T, uint32_t, VEC, kU>(rp, int(gz - ga), a.n_cls, s_c64, s_chi, s_clo, gather, acc);
        else
          state_sum<T, uint16_t, VEC, kU>(rp, int(gz - ga), a.n_cls, s_c64, s_chi, s_clo, gather, acc);
        T out[VEC];
        if (PASS_A) {
          const uint64_t w = __ldg(a.words + k);
          const uint32_t up = uint32_t(w >> a.n_sites), dn = uint32_t(w) & half;
          T xk[VEC], yk[VEC];
          if (staged) {
#pragma unroll
            for (int u = 0; u < VEC; ++u) xk[u] = xs[int(k - sb) * ncp + col0 + u];
          } else {
            C::load(x + int64_t(k) * ldx + col0, cvalid, xk);
          }
          C::load(y + int64_t(k) * ld + col0, cvalid, yk);
          const Coef<T> dc = diag_of<T>(hp, s_dhi, s_dlo, s_d64, up, dn);
#pragma unroll
          for (int u = 0; u < VEC; ++u) {
            acc[u].fma(dc.hi, dc.lo, xk[u]);
            out[u] = acc[u].value() + yk[u];
          }
          C::store(y + int64_t(k) * ld + col0, cvalid, out);
        } else {
#pragma unroll
          for (int u = 0; u < VEC; ++u) out[u] = acc[u].value();
          C::store(y + int64_t(__ldg(a.perm + k)) * ld + col0, cvalid, out);
        }
      }
    }
  }
}

// X in the dn-major order: xb[k][:] = x[perm[k]][:] (ncp columns per row of xb,
// VEC-column chunks; the padding columns of xb are zero)
template <typename T, int VEC>
__global__ void permute_rows_kernel(const T* __restrict__ x, int ld, int ncols, int ncp,
                                    const uint32_t* __restrict__ perm, int64_t n, T* __restrict__ xb) {
  using C = ChunkOf<T, VEC>;
  const int chunks = ncp / VEC;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n * chunks) return;
  const int64_t k = i / chunks;
  const int col0 = int(i % chunks) * VEC;
  T v[VEC];
  C::load(x + int64_t(__ldg(perm + k)) * ld + col0, ncols - col0, v);
  C::store(xb + k * ncp + col0, ncp - col0, v);
}

template <typename T, int VEC, int G>
cudaError_t launch_cached(mcd_ctx* c, const void* x, void* y, int ncols, int ld) {
  const int chunks = (ncols + VEC - 1) / VEC;
  const int ncp = chunks * VEC;
  const int off_xs = cls_bytes(c);
  const int smem = off_xs + kMStageBytes;
  static std::atomic<int> configured{-1};   // per instantiation
  if (configured < smem) {
    cudaFuncSetAttribute(hv_item_kernel<T, VEC, G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(hv_item_kernel<T, VEC, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    configured = smem;
  }
  // pass B reads X in the dn-major order, copied once (rows contiguous like pass A's)
  ConnCache& cb = c->idx.B.cc;
  const int64_t n = c->idx.n;
  const bool permuted = G > 1 && n > 0;
  if (permuted) {
    cudaError_t e = grow_bytes(cb.xbm, cb.xbm_cap, n * ncp * int64_t(sizeof(T)), c->stream);
    if (e != cudaSuccess) return e;
  }
  for (int pass = 0; pass < 2; ++pass) {
    const Layout& L = pass == 0 ? c->idx.B : c->idx.A;
    CArgs a;
    fill_args(c, L, a);
    a.x = x;
    a.y = y;
    a.ncols = ncols;
    a.ld = ld;
    a.ncp = ncp;
    if (pass == 0 && permuted) {
      const int64_t work = n * (ncp / VEC);
      permute_rows_kernel<T, VEC><<<int((work + 255) / 256), 256, 0, c->stream>>>(
          static_cast<const T*>(x), ld, ncols, ncp, L.perm, n, static_cast<T*>(cb.xbm));
      MCD_LAUNCHED(c);
      a.x = cb.xbm;
      // rows of the copy are ncp elements apart (the kernel's ldx); y keeps ld
      a.x_layout = 1;
    }
    a.off_xs = off_xs;
    a.xs_cap = int(kMStageBytes / sizeof(T));
    if (a.n_items <= 0) continue;
    timing_begin(c, pass == 0 ? 0 : 1);
    if (pass == 0)
      hv_item_kernel<T, VEC, G, false><<<int(a.n_items), kCT, smem, c->stream>>>(a, *c->hp);
    else
      hv_item_kernel<T, VEC, G, true><<<int(a.n_items), kCT, smem, c->stream>>>(a, *c->hp);
    MCD_LAUNCHED(c);
    timing_end(c);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T, int VEC>
cudaError_t dispatch_cols(mcd_ctx* c, const void* x, void* y, int ncols, int ld, bool* used) {
  const int chunks = (ncols + VEC - 1) / VEC;
  *used = true;
  if (chunks <= 1) return launch_cached<T, VEC, 1>(c, x, y, ncols, ld);
  if (chunks <= 2) return launch_cached<T, VEC, 2>(c, x, y, ncols, ld);
  if (chunks <= 4) return launch_cached<T, VEC, 4>(c, x, y, ncols, ld);
  if (chunks <= 6) return launch_cached<T, VEC, 6>(c, x, y, ncols, ld);
  if (chunks <= 8) return launch_cached<T, VEC, 8>(c, x, y, ncols, ld);
  if (chunks <= 12) return launch_cached<T, VEC, 12>(c, x, y, ncols, ld);
  if (chunks <= 16) return launch_cached<T, VEC, 16>(c, x, y, ncols, ld);
  *used = false;
  return cudaSuccess;
}

}  // namespace

cudaError_t cache_apply_items(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, bool* used) {
  *used = false;
  const bool f64 = dtype == MCD_F64;
  const int vec = f64 ? 2 : 4;
  const bool vec_ok = ncols >= 2 && ld % vec == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0 &&
                      reinterpret_cast<uintptr_t>(y) % 16 == 0;
  if (!vec_ok) return cudaSuccess;
  return f64 ? dispatch_cols<double, 2>(c, x, y, ncols, ld, used) : dispatch_cols<float, 4>(c, x, y, ncols, ld, used);
}

cudaError_t cache_items_prepare(mcd_ctx* c, int ncols, int dtype) {
  const int vec = dtype == MCD_F64 ? 2 : 4;
  const int64_t ncp = (ncols + vec - 1) / vec * vec;
  ConnCache& cb = c->idx.B.cc;
  return grow_bytes(cb.xbm, cb.xbm_cap, c->idx.n * ncp * (dtype == MCD_F64 ? 8 : 4), c->stream);
}

}  // namespace mcd
