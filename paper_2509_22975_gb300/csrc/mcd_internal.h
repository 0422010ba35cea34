// Internal declarations of the MCD library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mcd.h"

namespace mcd {

constexpr int kMaxSites = 32;
constexpr int kMaxBonds = kMaxSites * (kMaxSites - 1) / 2;   // 496
constexpr int kItem = 1024;          // states per work item of the block kernels
constexpr int kStageWords = 12288;   // minor words a CTA stages in shared memory
constexpr int kTimingClasses = 4;
constexpr int kMaxClasses = 16;      // distinct hopping amplitudes handled by class sums
constexpr int kMaxPClasses = 32;     // partner classes of the single-column kernel
constexpr int kMaxHopGroups = 64;    // (amplitude, j - i) groups of the hash kernel

// One undirected bond (i < j, t_ij != 0).  A state of one spin can hop along
// it iff exactly one of its two sites is occupied; the hop flips both bits.
struct Bond {
  uint32_t mask;      // (1 << i) | (1 << j)
  uint32_t between;   // sites strictly between i and j
  double t;           // t_ij
  float t_hi, t_lo;   // t_ij split into two floats (t_hi + t_lo == t to ~2^-48)
};

// Hamiltonian data passed to kernels by value (kernel parameter space).
struct HamParams {
  int n_sites;
  int n_bonds;
  int uniform;          // 1: diagonal = dtab[popc(up & dn)]
  int pad;
  double dtab[kMaxSites + 1];       // uniform diagonal by double occupancy
  float dtab_hi[kMaxSites + 1];
  float dtab_lo[kMaxSites + 1];
  const double* eps;    // device [n] (non-uniform case)
  const double* U;      // device [n] (non-uniform case)
  // Bonds are stored grouped by equal t_ij ("classes"): class c holds bonds
  // [c ? cls_end[c-1] : 0, cls_end[c]).  n_class = 0 when there are more than
  // kMaxClasses distinct amplitudes.
  int n_class;
  int cls_end[kMaxClasses];
  float cls_hi[kMaxClasses], cls_lo[kMaxClasses];
  double cls_t[kMaxClasses];
  Bond bonds[kMaxBonds];
  // Partner classes (n_sites <= 16): the bonds of one amplitude split into
  // classes in which every site is the first endpoint of at most one bond.
  // For class c, P_c(m) has bit i = bit partner_c(i) of m, so
  // (m ^ P_c(m)) & pfirst[c] marks the active bonds of c by their first
  // endpoint.  ppart[c] packs partner_c(i) in nibble i; pcls_t* is the common
  // amplitude of class c.  ptab (device) holds, for each group of four classes
  // and each byte position k in {0, 1} and byte value v, the four 16-bit
  // contributions of that byte to P_{4g..4g+3}(m), as one uint2.
  int n_pcls;                       // 0 = not available (n_sites > 16 or too many)
  uint32_t pfirst[kMaxPClasses];
  uint64_t ppart[kMaxPClasses];
  float pcls_hi[kMaxPClasses], pcls_lo[kMaxPClasses];
  double pcls_t[kMaxPClasses];
  const uint2* ptab;                // device [ceil(n_pcls / 4)][2][256]
  const uint2* pflip;               // device [n_pcls][16]: (flip, between) of first endpoint i
  // Hop groups (any n_sites): bonds (i, i + s) of one amplitude and one index
  // distance s.  For group g, hg_mask[g] has bit i set for each of its bonds,
  // so hg_mask[g] & (m ^ (m >> hg_shift[g])) marks the bonds of g along
  // which a spin word m can hop (exactly one endpoint occupied).
  int n_hg;                         // 0 = more than kMaxHopGroups groups
  uint32_t hg_mask[kMaxHopGroups];
  int hg_shift[kMaxHopGroups];
  float hg_hi[kMaxHopGroups], hg_lo[kMaxHopGroups];
  double hg_t[kMaxHopGroups];
};

// Work item of the hash kernel (hv_hash.cu): layout positions [s0, s1).
// log2p == 0: whole blocks [b0, b1) whose minor words the CTA hashes in
// shared memory.  Otherwise a chunk of the single block b0 (b1 = b0 + 1),
// looked up in that block's table of 2^log2p slots at htab + tab_off, or by
// binary search when log2p == kHashSearch (block too large for 16-bit slots).
// Every tabled block also has a one-bit-per-hash membership filter, so most
// absent targets are rejected by one load.
struct HItem {
  uint32_t s0, s1, b0, b1;
  uint32_t tab_off, log2p;
  uint32_t flt_off, log2f;   // membership filter of 2^log2f bits at hflt + flt_off
};
constexpr uint32_t kHashSearch = 0xFFu;


// One of the two orderings of the basis used by the H*v kernels.
//   up-major (A): basis order; blocks share an up word; minor = dn word.
//   dn-major (B): stable order by dn word; blocks share a dn word; minor = up.
// Work item of the connection cache (hv_cache.cu): layout positions [lo, hi)
// of the blocks b0..b1; every hop target of its states lies in the stage
// range [blk_off[b0], blk_off[b1 + 1]), and a record holds the target's
// position relative to blk_off[b0].  Its states, sorted by their number of
// records (most first, ties in position order), form slices of 32, numbered
// from slice0; flags bit 0 = 4-byte records.  sb, se = its stage range,
// g0, g1 = its record groups [g0, g1) (filled once the records are laid out).
struct CItem {
  uint32_t lo, hi, b0, b1, slice0, flags, sb, se, g0, g1;
};

// Connection cache of one layout: the found hops of every state of the
// pass, as records in slices of 32 states.  smap[32 s + l] is the state of
// lane l of slice s (position relative to its item's lo; 0xFFFF = none).
// Record group g (256 bytes) of a slice holds 8 bytes per lane: the next
// 16 / record-size records of the lane's state, padded with all-ones
// records.  col[s] is the first group of slice s (col[n_slices] = total).
// Records: 2 bytes = pos:14 | sign:1 | class:1, or 4 bytes = pos:22 |
// sign:1 | class:9; class indexes the coefficient tables (amplitude classes,
// or bonds when there is no class table).
struct ConnCache {
  int valid = 0;                 // built for the current basis and Hamiltonian
  int failed = 0;                // cannot be built for them (auto mode falls back)
  int rec_bytes = 0;             // 2 (some items may hold 4-byte records) or 4 (all)
  int n_cls = 0;
  int64_t n_items = 0, n_slices = 0, n_groups = 0;
  int64_t max_stage = 0;         // largest stage range of an item (states)
  int64_t n_conn = 0;            // found hops (records that are not padding)
  CItem* items = nullptr;
  uint32_t* col = nullptr;       // [n_slices + 1]
  uint16_t* smap = nullptr;      // [n_slices * 32]
  void* rec = nullptr;           // [n_groups * 256 bytes]
  double* c64 = nullptr;         // [n_cls] coefficient
  float* chi = nullptr;          // [n_cls] coefficient split in two floats
  float* clo = nullptr;
  void* xb = nullptr;            // x in this layout's order (streaming kernel of pass B)
  void* xbm = nullptr;           // X (many columns) in this layout's order (pass B)
  void* yb = nullptr;            // pass B's part of y (streaming kernels), read by pass A
  unsigned int* err = nullptr;   // set by a kernel whose bounded wait ran out
  unsigned int* sched = nullptr; // streaming kernel's item counter and CTA ticket (zero between launches)
  int64_t items_cap = 0, col_cap = 0, smap_cap = 0, rec_cap = 0, cls_cap = 0, xb_cap = 0, yb_cap = 0, xbm_cap = 0;
  // many-column kernel: work units (items of one stage range, column tile)
  // of the last column count and element size (the items' stage ranges are
  // kept on the host in mcd_ctx::stage_range)
  uint4* units = nullptr;
  int64_t n_units = 0, units_cap = 0;
  int units_key = -1;            // ncp * 16 + element size of `units` (-1 none)
};

struct Layout {
  int64_t n = 0;
  int64_t nblk = 0;
  int64_t n_items = 0;
  uint32_t* minor = nullptr;     // [n]
  uint32_t* blk_off = nullptr;   // [nblk + 1]
  uint32_t* blk_major = nullptr; // [nblk]
  uint32_t* item_blk = nullptr;  // [n_items + 1] block of the first state of item i
  uint32_t* perm = nullptr;      // [n] layout position -> basis index (B only)
  // hash-kernel work items and per-block tables (built on first use)
  int hash_built = 0;            // item size they were built for (0 = none)
  int64_t n_hitems = 0;
  int64_t hitem_cap = 0;
  HItem* hitems = nullptr;
  int64_t htab_len = 0;
  int64_t htab_cap = 0;
  uint32_t* htab = nullptr;
  int64_t hflt_len = 0;          // 32-bit words
  int64_t hflt_cap = 0;
  uint32_t* hflt = nullptr;
  ConnCache cc;                  // found hops of every state (hv_cache.cu)
};

struct DevIndex {
  int64_t n = 0;
  int64_t cap = 0;               // states the buffers below can hold
  uint64_t* words = nullptr;     // [n] basis words (device)
  Layout A, B;
  int64_t nnz = -1;              // off-diagonal nonzeros (lazy)
};

struct LanczosWork {
  int64_t n = 0;
  int dtype = -1;
  void* W = nullptr;             // H s_n
  void* V = nullptr;             // Krylov vectors: nvec slots of ld elements
  int64_t ld = 0;                // slot stride: n rounded up to 4 (16-byte aligned slots)
  int nvec = 0;                  // max_iter + 1 (all stored) or 2 (rotating)
  bool stored = false;
  double* psi64 = nullptr;       // fp64 Ritz vector and H psi (fp32 form polish)
  double* w64 = nullptr;
  double* coef = nullptr;        // device Ritz coefficients
  double* scal = nullptr;        // device scalar area (see krylov.cu)
  int scal_cap = 0;
  double* partials = nullptr;    // per-CTA fp64 partial sums
  unsigned int* ticket = nullptr;
  int max_ctas = 0;
};

struct Timing {
  cudaEvent_t ev[2 * 1024];
  int n_ev = 0;
  int cls[1024];
  double ms[kTimingClasses] = {0, 0, 0, 0};
  int64_t count[kTimingClasses] = {0, 0, 0, 0};
  bool created = false;
};

}  // namespace mcd

struct mcd_ctx {
  int device = -1;
  cudaStream_t stream = nullptr;
  std::string err;
  // Hamiltonian
  bool has_ham = false;
  int n = 0, n_up = 0, n_dn = 0;
  std::vector<double> t, eps, U;
  mcd::HamParams* hp = nullptr;       // host copy (large struct)
  double* d_eps = nullptr;
  double* d_U = nullptr;
  void* d_pclass = nullptr;           // partner-class tables (pt, pe)
  // Basis (host copy valid when basis_on_host; n_basis is authoritative)
  std::vector<uint64_t> basis;
  int64_t n_basis = 0;
  bool basis_on_host = false;
  int64_t launches = 0;
  mcd::DevIndex idx;
  // Krylov
  mcd::LanczosWork lw;
  double* gs_psi = nullptr;            // normalised ground state (fp64, device)
  int64_t gs_n = 0;
  double gs_E0 = 0.0;
  bool gs_valid = false;
  std::vector<double> last_a, last_b;
  // Options
  int hv_algo = 0;
  int hash_item = 1024;                // states per work item of the hash kernel
  int timing = 0;
  int sampler_threads = 0;
  int sampler_where = 0;                // 0 auto, 1 host threads, 2 device
  int hv_cache = 0;                     // 0 auto, 1 off, 2 required
  std::vector<uint2> stage_range[2];    // connection cache: stage range {sb, se} of each item, layouts B and A
  int krylov_store = 0;                 // 0 auto, 1 always regenerate the Lanczos vectors
  int apply_sync = 1;                   // mcd_apply waits and reads the wait-error words
  int hv_cols = 0;                      // many-column kernel: 0 timed pick, 1 pipelined tiles, 2 CTA per item
  int batch_split = 0;                  // batched H*v: parts per work item (0 timed, 1, 2 or 4)
  int batch_mode = 0;                   // batched Lanczos: 0 per-instance solves on a stream pool, 1 lockstep launches
  bool keep_gs = false;                 // Lanczos forms the Ritz vector (kept for the Green function) even
                                        // without a caller's psi (set by the batched solves)
  int cols_pick[65][2] = {};            // timed pick per column count (<= 64) and dtype: 0 none, 1 tiles, 2 items
  cudaEvent_t tune_ev[3] = {nullptr, nullptr, nullptr};
  int64_t wait_test_item = -1;          // one-shot: withhold this item's copies (time-out test)
  mcd::Timing* tm = nullptr;
  bool tm_borrowed = false;             // tm belongs to another context (band Lanczos runs)
};

namespace mcd {


// streaming multiprocessors of the current device (queried once per device)
int device_sms();

// error helpers (mcd_api.cu)
int fail(mcd_ctx* c, int status, const std::string& msg);
int cuda_fail(mcd_ctx* c, cudaError_t e, const char* where);

// host sampler (sampler.cpp)
int sample_basis(mcd_ctx* c, uint64_t seed, int64_t n_target, double beta,
                 const uint64_t* seeds, int64_t n_seed, int flags,
                 std::vector<uint64_t>& out);
double sector_size(int n, int n_up, int n_dn);

// host eigensolvers (tridiag.cpp, symeig.cpp)
double tridiag_lowest(const double* a, const double* b, int m, double* vec /*nullable [m]*/);
// eigenvalues w[n] ascending of symmetric A (row-major n x n, destroyed) and the
// leading `rows` rows of the eigenvector matrix X[rows][n]; 0 on success
int symeig_leading(int n, double* A, double* w, int rows, double* X);

// adjoint of H*v with respect to (t, eps, U) (adjoint.cu)
int hv_adjoint(mcd_ctx* c, const void* u, const void* v, int ncols, int ld, int dtype, double* grad_t,
               double* grad_eps, double* grad_U);

// band Lanczos Green function (band.cu)
int band_lanczos_green(mcd_ctx* c, const int* site, const int* spin, int L, int n_blocks, double w_t, int dtype,
                       const double* z_re, const double* z_im, int nz, double* G_re, double* G_im,
                       int64_t* dim_plus, int64_t* dim_minus);

// device sampler (sampler_gpu.cu): same result as sample_basis; applies when
// every nonzero U_i has the same value; installs the basis on the device
bool device_sampler_eligible(const mcd_ctx* c);
// keys[0, n) sorted in place on their low `bits` bits, *out = the distinct
// keys in ascending order (*nout of them; stream-ordered allocation on the
// context's stream that the caller frees with cudaFreeAsync)
int sort_unique_device(mcd_ctx* c, uint64_t* keys, int64_t n, int bits, uint64_t** out, int64_t* nout);
int sample_basis_device(mcd_ctx* c, uint64_t seed, int64_t n_target, double beta, const uint64_t* seeds,
                        int64_t n_seed, int flags, int64_t* n_out);

// batches of contexts (batch.cu)
int batch_apply(mcd_ctx* const* ctxs, int n, const void* x, void* y, int dtype);
int batch_lanczos_ground(mcd_ctx* const* ctxs, int n, int max_iter, double tol, uint64_t seed, int dtype,
                         double* E0, int* iters, double* resid, void* const* psi);

// gradient of the Green function (band.cu)
int green_gradient(mcd_ctx* c, const int* site, const int* spin, int L, int n_blocks, double w_t,
                   const double* z_re, const double* z_im, int nz, const double* g_re, const double* g_im,
                   double* grad_t, double* grad_eps, double* grad_U, double cg_tol, int* cg_iters);

// device index (index.cu)
int build_index(mcd_ctx* c, const uint64_t* words, int64_t n, bool on_device);
// exclusive scan of n uint32 values (in may equal out), stream-ordered
cudaError_t scan_u32(mcd_ctx* c, const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);
void free_index(DevIndex& ix, cudaStream_t s);   // stream-ordered frees on s

// H*v (hv.cu)
int hv_apply(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype,
             double* dot_partials, int dot_slot);
int hv_diagonal(mcd_ctx* c, double* out);
int hv_connections(mcd_ctx* c, int64_t* rows, int64_t* cols, double* vals, int64_t cap,
                   int64_t* nnz);
int hv_dot_ctas(mcd_ctx* c, int ncols, int dtype);

// hash-lookup H*v (hv_hash.cu): used for n_sites > 16 (or when forced by
// MCD_OPT_HV_ALGO); both passes, fused <x, y> when dot_out is given
bool hash_eligible(const mcd_ctx* c);
int hash_apply(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, double* dot_partials,
               int max_parts, unsigned int* ticket, double* dot_out);
void free_hash(Layout& L, cudaStream_t s);

// connection cache (hv_cache.cu): built by the first H*v of a basis (when
// c->hv_cache allows and hv_algo == 0), then used by every H*v whose columns
// it covers; returns MCD_OK and sets *used when it applied y = H~ x
int cache_apply(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, double* dot_partials,
                int max_parts, unsigned int* ticket, double* dot_out, bool* used);
void cache_invalidate(Layout& L);
void free_cache(Layout& L, cudaStream_t s);
// *out = 1 when a bounded wait of a cached kernel gave up since the records were built
int cache_errors(mcd_ctx* c, unsigned int* out);
// MCD_E_TIMEOUT (and the words cleared) when a bounded wait gave up since the
// last check, else MCD_OK; synchronizes the context's stream
int take_wait_errors(mcd_ctx* c);
// cached H*V for many columns, or one column with a row stride (hv_cache_cols.cu);
// *used = false when the columns' layout is not covered (the caller falls back)
cudaError_t cache_apply_cols(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, bool* used);
// the CTA-per-item many-column kernel (hv_cache_items.cu) and its scratch
cudaError_t cache_apply_items(mcd_ctx* c, const void* x, void* y, int ncols, int ld, int dtype, bool* used);
cudaError_t cache_items_prepare(mcd_ctx* c, int ncols, int dtype);

// Lanczos (krylov.cu)
int lanczos_ground(mcd_ctx* c, int max_iter, double tol, uint64_t seed, int dtype,
                   double* E0, void* psi, int* iters, double* residual);
void free_lanczos(LanczosWork& w);
// *out (device) = sum_k a[k] b[k] over n elements of dtype, fixed-order reduction
int vec_dot(mcd_ctx* c, const void* a, const void* b, int64_t n, int dtype, double* out);

// timing helpers (hv.cu)
void timing_begin(mcd_ctx* c, int cls);
void timing_end(mcd_ctx* c);
void timing_collect(mcd_ctx* c);

}  // namespace mcd

// count one kernel launch of context c
#define MCD_LAUNCHED(c) (++(c)->launches)
