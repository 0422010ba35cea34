/*
 * mcd.h -- C ABI of the Monte Carlo diagonalization hot path on one GB300.
 *
 * The library applies the Hubbard Hamiltonian (Eq. (1) of arXiv 2509.22975,
 * generalised to hoppings t_ij, on-site energies eps_i and repulsions U_i)
 * projected onto a truncated basis F~ of Fock states (Sec. "Subspace of the
 * ground state", the Eq. defining H~_mn = <x~_m|H|x~_n>), without storing the
 * matrix (App. B), and runs the Lanczos ground-state recursion (App. B) on it.
 *
 * Conventions
 *   - Fock state word: w = (up << n_sites) | dn, bit i of each half = site i
 *     (App. D: |90> = |0101;1010>, spin up in the high half).  n_sites <= 32.
 *   - Fermionic mode order: up modes 0..n-1, then down modes 0..n-1.  A hop
 *     c^dag_{i s} c_{j s} has sign (-1)^(occupied same-spin sites strictly
 *     between i and j).
 *   - A basis is a strictly ascending array of words of one (N_up, N_dn)
 *     sector, at most 2^31 - 1 states.
 *   - Vectors over the basis are row-major [n_states][ld] blocks of ncols <= ld
 *     columns, in basis order, on the device of the context.
 *
 * Ownership: the caller owns every pointer it passes; host arrays are copied
 * in before the call returns; device arrays are only used during the call,
 * on the context's stream.  The context owns its Hamiltonian, basis, index
 * and Krylov workspace and frees them in mcd_destroy.
 *
 * Errors: every entry point returns an mcd_status; negative values are
 * errors and leave the context usable; mcd_last_error() describes the last
 * failure of that context.  Positive values are warnings.  No exceptions
 * cross the ABI.  A context is not thread-safe: use one per host thread.
 */
#ifndef MCD_H
#define MCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcd_ctx mcd_ctx;

typedef enum {
  MCD_OK = 0,
  MCD_W_SHORT = 1,            /* sampler stopped with fewer states than asked */
  MCD_E_INVALID = -1,         /* bad argument, unsorted/duplicate basis, ... */
  MCD_E_SECTOR = -2,          /* word or seed outside the (N_up, N_dn) sector */
  MCD_E_OOM = -3,             /* host or device allocation failed */
  MCD_E_CUDA = -4,            /* a CUDA call failed (message in last_error) */
  MCD_E_NOT_CONVERGED = -5,   /* Lanczos hit max_iter above tolerance */
  MCD_E_BREAKDOWN = -6,       /* non-finite Lanczos coefficient */
  MCD_E_TIMEOUT = -7,         /* a bounded device wait gave up: the product is incomplete */
  MCD_E_STATE = -8,           /* call out of order (no Hamiltonian / basis) */
  MCD_E_NODEVICE = -9         /* device work asked of a host-only context */
} mcd_status;

typedef enum { MCD_F64 = 0, MCD_F32 = 1 } mcd_dtype;

/* Sampler flags (mcd_build_basis). */
#define MCD_SAMPLE_NEW_ONLY 1   /* next starting points = new states only */

/* Options (mcd_set_option). */
#define MCD_OPT_HV_ALGO 1       /* 0 = two-layout block kernels, in-block
                                   lookup by shared bitmap when n_sites <= 16,
                                   by hash table otherwise (default);
                                   1 = plain per-state global binary search;
                                   2 = two-layout block kernels, binary search;
                                   3 = two-layout block kernels, hash lookup
                                   at any n_sites */
#define MCD_OPT_KERNEL_TIMING 2 /* 1 = record CUDA events around H*v launches */
#define MCD_OPT_SAMPLER_THREADS 3 /* host threads of the sampler (0 = auto)  */
#define MCD_OPT_SAMPLER_DEVICE 5 /* where mcd_build_basis runs: 0 = on the
                                   context's GPU when it has one and every
                                   nonzero U_i has the same value, else on
                                   host threads (default); 1 = host threads;
                                   2 = GPU (MCD_E_INVALID when not possible).
                                   Both give the same basis, word for word. */
#define MCD_OPT_HV_CACHE 6       /* connection cache of H*v: 0 = the first
                                   H*v of a basis (and Hamiltonian) runs the
                                   matrix-free enumeration and lookup once and
                                   keeps the found hops in device memory
                                   (2 or 4 bytes each), later H*v stream them,
                                   when they fit in half the free memory
                                   (default); 1 = off (every H*v enumerates
                                   and looks up, nothing stored); 2 = required
                                   (mcd_apply fails when the records cannot be
                                   built).  Only with MCD_OPT_HV_ALGO = 0.
                                   The result is the same matrix, summed in
                                   another order (within rounding). */
#define MCD_OPT_APPLY_SYNC 7     /* 1 = mcd_apply waits for its product and
                                   returns MCD_E_TIMEOUT when a bounded wait
                                   of the streaming kernel gave up (default);
                                   0 = mcd_apply returns after the launch and
                                   such a failure is reported by the next call
                                   that reads it (mcd_apply with 1,
                                   mcd_lanczos_ground, mcd_band_lanczos_green,
                                   mcd_hv_cache_info).  A reported failure is
                                   cleared, so later calls can succeed. */
#define MCD_OPT_WAIT_TEST 8      /* test of the time-out path: value k >= 0
                                   makes the next cached product withhold the
                                   arrival that completes the shared-memory
                                   stage of work item k (one column) or work
                                   unit k (many columns) of its second pass
                                   and poll each wait only 4096 times, so that
                                   the waits on it give up; -1 = off (default).
                                   Applies to one product, then resets. */
#define MCD_OPT_KRYLOV_STORE 9   /* Lanczos vectors of mcd_lanczos_ground:
                                   0 = kept in device memory when they fit in
                                   half of the free memory, else regenerated
                                   (default); 1 = always regenerated: two
                                   rotating slots, and a second pass of the
                                   recursion (same fixed-order reductions, so
                                   the same vectors bit for bit) forms the
                                   Ritz vector. */
#define MCD_OPT_HV_COLS 10       /* cached H*V with several columns: 0 = the
                                   first product of each column count (<= 64)
                                   and dtype of a basis and Hamiltonian times
                                   both kernels (pipelined column tiles, CTA
                                   per work item) and later products use the
                                   faster (default); 1 = pipelined tiles;
                                   2 = CTA per work item.  Same matrix, summed
                                   in another order (within rounding). */
#define MCD_OPT_BATCH_SPLIT 11   /* batched calls (mcd_batch_*), read from
                                   the first context: states per work unit of
                                   the batched H*v are 1024 / value; 0 = the
                                   first product of each batch size class
                                   times value 1, 2 and 4 with 2, 4 and 8 CTAs
                                   per SM and keeps the fastest (default).
                                   Products are the same bit for bit for
                                   every value; the Lanczos scalars <v, Hv>
                                   are summed in another order (within
                                   rounding). */
#define MCD_OPT_BATCH_MODE 12   /* mcd_batch_lanczos_ground, read from the
                                   first context: 0 = every instance's own
                                   solve (mcd_lanczos_ground, with its
                                   connection cache) on a pool of host
                                   threads, each with its own stream: the
                                   results of separate calls, bit for bit
                                   (default); 1 = one sequence of launches
                                   over all instances in lockstep (the
                                   matrix-free batched H*v, CUDA-graph
                                   replay; instances of one site count). */
#define MCD_OPT_HASH_ITEM 4     /* states per work item of the hash-lookup
                                   kernels: a power of two in [64, 4096]
                                   (default 1024).  Blocks of more states are
                                   split into items that share one table of
                                   the block in device memory. */

/* Create a context on CUDA device `device` using `cuda_stream` (a
 * cudaStream_t, may be NULL for the legacy default stream).  device = -1
 * makes a host-only context: Hamiltonian, sampler and basis calls work, every
 * device call returns MCD_E_NODEVICE.  *out is NULL on failure. */
int mcd_create(mcd_ctx** out, int device, void* cuda_stream);
int mcd_destroy(mcd_ctx* ctx);
int mcd_set_stream(mcd_ctx* ctx, void* cuda_stream);
int mcd_set_option(mcd_ctx* ctx, int option, int64_t value);
/* Message of the last failure of ctx ("" if none).  Valid until the next call
 * on ctx.  ctx may be NULL (then a static message about creation). */
const char* mcd_last_error(const mcd_ctx* ctx);
const char* mcd_status_string(int status);

/* Eq. (1): H = sum_{i!=j,s} t[i*n+j] c^dag_{is} c_{js} + sum_{i,s} eps[i] n_{is}
 *            + sum_i U[i] n_{i,up} n_{i,dn}.
 * t: host [n*n] real, must be symmetric (else MCD_E_INVALID), diagonal
 * ignored.  eps: host [n] or NULL (zero; the paper's -mu goes here).
 * U: host [U_len] with U_len = 1 (uniform) or n.  1 <= n <= 32,
 * 0 <= n_up, n_dn <= n.  Replaces any previous Hamiltonian and drops the
 * basis if the sector changes. */
int mcd_set_hamiltonian(mcd_ctx* ctx, int n_sites, const double* t, const double* eps,
                        const double* U, int U_len, int n_up, int n_dn);

/* Sec. "Subspace of the ground state": grow F~ from the seed words by steps,
 * proposing every hopping term of every starting state and accepting a
 * proposed state b with probability min(exp(-beta sum_i U_i n_i,up n_i,dn(b)), 1).
 * Random draws: one uniform number per proposal from SplitMix64 (its
 * published output function), keyed by (seed, step, parent word, hop id), so
 * the draws do not depend on where or in which order proposals are made.
 * seed_states: host [n_seed] >= 1 words of the sector.  Stops at exactly
 * n_target states (a final overshooting step keeps the new states of smallest
 * SplitMix64 priority), or earlier if no new state appears for 64 steps
 * (returns MCD_W_SHORT).  n_target must not exceed the sector size.  The basis
 * replaces the current one and is indexed on the device (if any). *n_out =
 * basis size.  Runs on the context's GPU or on host threads
 * (MCD_OPT_SAMPLER_DEVICE, MCD_OPT_SAMPLER_THREADS); every placement and thread
 * count gives the same words. */
int mcd_build_basis(mcd_ctx* ctx, uint64_t seed, int64_t n_target, double beta,
                    const uint64_t* seed_states, int64_t n_seed, int flags, int64_t* n_out);

/* Install a basis given as host words (strictly ascending, all in the sector;
 * anything else is MCD_E_INVALID / MCD_E_SECTOR, nothing is sorted silently)
 * and build its device index. n >= 1.  With a device the words are copied to
 * it as they are and checked there (pinned host memory makes the copy a
 * direct DMA); a host-only context checks and keeps them on the host.  The
 * caller's array is not referenced after the call returns. */
int mcd_set_basis(mcd_ctx* ctx, const uint64_t* host_words, int64_t n);
/* Same as mcd_set_basis for words already in device memory (dev_words[n] on
 * the context's device).  Order and sector are checked on the device; the
 * words are copied (the caller keeps ownership). */
int mcd_set_basis_device(mcd_ctx* ctx, const uint64_t* dev_words, int64_t n);
/* Copy the basis to host_out[cap]; *n = basis size (also when cap is short). */
int mcd_get_basis(const mcd_ctx* ctx, uint64_t* host_out, int64_t cap, int64_t* n);
/* Basis file (checkpoint of a sampled truncated basis F~, Sec. "Subspace of
 * the ground state"): mcd_save_basis writes the installed basis to path as a
 * 40-byte little-endian header (magic "MCDBASIS", version 1, n_sites, N_up,
 * N_dn as uint32, N_f as int64, FNV-1a 64-bit hash of the words' bytes)
 * followed by the N_f uint64 words; MCD_E_STATE without a Hamiltonian or a
 * basis, MCD_E_INVALID if the file cannot be written.  mcd_load_basis reads
 * such a file and installs it as mcd_set_basis would: MCD_E_STATE without a
 * Hamiltonian, MCD_E_SECTOR if the file's sector differs from the
 * Hamiltonian's, MCD_E_INVALID for a missing, short, foreign or corrupted file
 * (magic, version, size or hash) and for words out of order.  A file
 * rejected before its words are checked (magic, version, sector, size, hash)
 * leaves the current basis in place.  path is a NUL-terminated file name, not
 * referenced after the call. */
int mcd_save_basis(const mcd_ctx* ctx, const char* path);
int mcd_load_basis(mcd_ctx* ctx, const char* path);
/* Sizes of the installed basis and its index; nnz_offdiag = number of nonzero
 * off-diagonal entries of H~ (counted on the device; pass NULL to skip). */
int mcd_basis_info(mcd_ctx* ctx, int64_t* n_states, int64_t* n_up_blocks,
                   int64_t* n_dn_blocks, int64_t* nnz_offdiag);

/* y = H~ x (App. B: targets outside F~ are discarded, i.e. the projected
 * matrix is applied).  x, y: device, dtype MCD_F64 or MCD_F32, row-major
 * [n_states][ld], ncols columns (1 <= ncols <= ld); x and y must not overlap.
 * FP32 vectors use fp64 hopping and diagonal coefficients (each split into
 * two floats) and accumulate each row in fp32. */
int mcd_apply(mcd_ctx* ctx, const void* x, void* y, int ncols, int ld, int dtype);

/* Adjoint of mcd_apply with respect to the parameters of Eq. (1): for device
 * blocks u, v (dtype, [n_states][ld], ncols columns), the derivatives of
 * <u, H~ v> = sum_c u[:, c]^T H~ v[:, c], accumulated in fp64:
 *   grad_t[i*n+j] = grad_t[j*n+i] = d/dt_ij for every bond with t_ij != 0
 *                   (one parameter per bond; 0 elsewhere),
 *   grad_eps[i]   = d/deps_i,   grad_U[i] = d/dU_i.
 * Host outputs, each nullable.  With u = v = |Omega~> these are the
 * Hellmann-Feynman derivatives of E0; the adjoint with respect to v is H~ u
 * (mcd_apply), H~ being symmetric. */
int mcd_hv_adjoint(mcd_ctx* ctx, const void* u, const void* v, int ncols, int ld, int dtype,
                   double* grad_t, double* grad_eps, double* grad_U);

/* Diagonal <x~_k|H|x~_k> of H~ in fp64, written to device diag_dev[n_states]. */
int mcd_diagonal(mcd_ctx* ctx, double* diag_dev);

/* Off-diagonal entries of H~ as (row, col, value = t_ij * sign) triples in
 * device arrays of capacity cap, grouped by row (order inside a row is not
 * specified).  *nnz = total count; with rows_dev == NULL only counts. */
int mcd_connections(mcd_ctx* ctx, int64_t* rows_dev, int64_t* cols_dev, double* vals_dev,
                    int64_t cap, int64_t* nnz);

/* No counterpart in the paper: the same output as mcd_connections, for
 * callers that must not allocate device memory (a caller whose memory is all
 * owned by its own pool, or one under a fixed memory budget where a late
 * allocation can fail).  The per-row counts and offsets live in one fixed
 * 2 MiB array of device global memory that the library defines, so this call
 * allocates nothing; every GPU that loads the library keeps that array until
 * the process exits.  Limit: bases of at most 262144 states, else
 * MCD_E_INVALID.  The first call on a device looks up the array's address and
 * keeps it (that first call should come before any stream capture; after a
 * cudaDeviceReset by the application the call is not supported).  All calls
 * share the array: calls whose work overlaps on the GPU race.  With rows_dev
 * set and cap < *nnz the call returns MCD_E_INVALID with *nnz set.  Entries
 * are grouped by row; their order inside a row differs from call to call. */
int mcd_connections_noalloc(mcd_ctx* ctx, int64_t* rows_dev, int64_t* cols_dev, double* vals_dev,
                            int64_t cap, int64_t* nnz);

/* App. B: Lanczos ground state of H~ from a SplitMix64 start vector keyed by
 * `seed`, normalised form of the recursion (a_n, b_n as in App. B), Krylov
 * vectors and H~ products in dtype, coefficients and the tridiagonal
 * eigenproblem in fp64.  Stops when the residual estimate b_{m} |s_{m-1}|
 * < tol * max(1, |E0|), on an invariant subspace (b < 1e-14 scale), or at
 * max_iter (then MCD_E_NOT_CONVERGED unless tol <= 0, which asks for exactly
 * max_iter steps).  The Krylov vectors are kept in device memory when they
 * fit in half of it (else regenerated by a second pass) to form the Ritz
 * vector sum_n |n><n|Omega_eff> (change-of-basis Eq. of App. B) in fp64.
 * dtype MCD_F64: E0 = lowest Ritz value.  dtype MCD_F32: E0 = the fp64
 * Rayleigh quotient <psi|H~|psi>/<psi|psi> of that Ritz vector (fp64 H~
 * product), which removes the fp32 recursion's error to first order.
 * psi_dev (nullable): device [n_states] of dtype, receives the normalised
 * Ritz vector.  *residual = |H~ psi - E0 psi| / |psi| when the Ritz vector was
 * formed (fp32 always, fp64 with psi_dev), else the estimate.  E0, iters,
 * residual: host. */
int mcd_lanczos_ground(mcd_ctx* ctx, int max_iter, double tol, uint64_t seed, int dtype,
                       double* E0, void* psi_dev, int* iters, double* residual);

/* Sec. "Subspace of the Green function", Sec. "Further truncation", App. C:
 * Green function of the ground state left by the last mcd_lanczos_ground
 * (which keeps its normalised Ritz vector and E0).  The ground state is
 * truncated to the shortest prefix of its largest |c_n|^2 (ties: lower index)
 * reaching w_t of its norm and renormalised; F~+ = U_mu c^dag_mu F~ and
 * F~- = U_mu c_mu F~; the start blocks c^dag_mu|Omega~>, c_mu|Omega~>; band
 * Lanczos (blocked H~V, fp64 Gram-Schmidt twice against the last two blocks,
 * rank-revealing Cholesky QR with deflation at 1e-10 (fp64) / 1e-5 (fp32) of a
 * column's norm) for n_block_iter blocks in each space; the eigenpairs of the
 * banded H_eff (fp64, host); Q = <phi_mu|E_m>; and
 *   G_{mu nu}(z) = sum_m Q+_{mu m} Q+_{nu m} / (z + E0 - E+_m)
 *                + sum_n Q-_{mu n} Q-_{nu n} / (z - E0 + E-_n).
 * orb_site, orb_spin: host [L], 1 <= L <= 64, one spin for all (G is block
 * diagonal in spin).  dtype: the Krylov vectors (MCD_F64 / MCD_F32).
 * z_re, z_im: host [nz] (z = omega + i eta, or i omega_n).  G_re, G_im: host
 * [nz][L][L].  dim_plus, dim_minus (nullable): |F~+|, |F~-|.  MCD_E_STATE
 * without a ground state. */
int mcd_band_lanczos_green(mcd_ctx* ctx, const int* orb_site, const int* orb_spin, int L,
                           int n_block_iter, double w_t, int dtype, const double* z_re,
                           const double* z_im, int nz, double* G_re, double* G_im,
                           int64_t* dim_plus, int64_t* dim_minus);

/* Gradient of the Green function with respect to the Hamiltonian's
 * parameters (for fitting bath parameters to a target G(i omega_n)), as a
 * vector-Jacobian product: the gradient of
 *   S = sum_{z, mu, nu} gG_re[z][mu][nu] Re G_mu nu(z) + gG_im[z][mu][nu] Im G_mu nu(z)
 * with G as mcd_band_lanczos_green computes it (same orbitals, n_block_iter,
 * w_t, z; fp64 Krylov vectors) and the set of kept ground-state words held
 * fixed.  Ingredients: Hellmann-Feynman dE0 = <Omega|dH|Omega>; the
 * first-order ground-state response (H - E0) dOmega = -(dH - dE0) Omega,
 * solved once for the contracted right-hand side by conjugate gradients
 * (relative residual cg_tol, e.g. 1e-11); the resolvent's derivative in each
 * excited space from the band run's Ritz vectors (all Krylov blocks are kept:
 * |F~+-| x n_block_iter x L doubles each, MCD_E_OOM if they do not fit).
 * grad_t: host [n][n] (bond derivative at [i][j] and [j][i], 0 off the
 * bonds); grad_eps, grad_U: host [n].  *cg_iters (nullable): CG iterations.
 * MCD_E_STATE without a ground state; MCD_E_NOT_CONVERGED if CG does not reach
 * cg_tol (gradients still filled). */
int mcd_green_gradient(mcd_ctx* ctx, const int* orb_site, const int* orb_spin, int L, int n_block_iter,
                       double w_t, const double* z_re, const double* z_im, int nz, const double* gG_re,
                       const double* gG_im, double cg_tol, double* grad_t, double* grad_eps, double* grad_U,
                       int* cg_iters);

/* App. C for many impurity models at once (the embedding use of the
 * method): for every instance i, mcd_band_lanczos_green on ctxs[i] (its
 * Hamiltonian, basis and the ground state left by mcd_lanczos_ground or
 * mcd_batch_lanczos_ground) with the same orbitals, n_block_iter, w_t, dtype
 * and z points.  G_re, G_im: host [n_inst][nz][L][L]; dim_plus, dim_minus:
 * host [n_inst] (nullable).  The instances run concurrently: a pool of host
 * threads, each with its own CUDA stream, takes instances one after another
 * (every buffer the calls allocate is stream-ordered, so they do not
 * synchronise the device); each context's stream is restored afterwards and
 * the results equal those of the one-instance call.  A context appears once.
 * Returns the first failing instance's status (its message, prefixed with its
 * index, in ctxs[0]'s last error). */
int mcd_batch_band_lanczos_green(mcd_ctx* const* ctxs, int n_inst, const int* orb_site, const int* orb_spin,
                                 int L, int n_block_iter, double w_t, int dtype, const double* z_re,
                                 const double* z_im, int nz, double* G_re, double* G_im, int64_t* dim_plus,
                                 int64_t* dim_minus);

/* mcd_green_gradient for many instances at once (gradients with respect to
 * each instance's bath and cluster parameters), run like
 * mcd_batch_band_lanczos_green.  Every instance has the same number of sites
 * n.  gG_re, gG_im: host [n_inst][nz][L][L]; grad_t: host [n_inst][n][n];
 * grad_eps, grad_U: host [n_inst][n]; cg_iters: host [n_inst] (nullable). */
int mcd_batch_green_gradient(mcd_ctx* const* ctxs, int n_inst, const int* orb_site, const int* orb_spin, int L,
                             int n_block_iter, double w_t, const double* z_re, const double* z_im, int nz,
                             const double* gG_re, const double* gG_im, double cg_tol, double* grad_t,
                             double* grad_eps, double* grad_U, int* cg_iters);

/* App. B/C (diagonalising the effective matrices): eigenvalues w[n]
 * (ascending) of the symmetric host matrix A[n][n] (row-major; not modified)
 * and the first `rows` rows of its eigenvector matrix X[rows][n] (column m =
 * eigenvector of w[m]; X may be NULL).  Householder tridiagonalisation and
 * implicit QR with the Wilkinson shift, fp64.  MCD_E_NOT_CONVERGED if the QR
 * iteration cap is reached. */
int mcd_symeig(int n, const double* A, double* w, int rows, double* X);

/* Batches of small models (embedding calculations: many impurity models,
 * each with its own Hamiltonian and Monte Carlo basis of its own size).
 * ctxs[n_inst]: contexts on one device, each with a Hamiltonian of at most 16
 * sites and an installed basis; they are read, not modified (except for
 * launch counts and error text, which go to ctxs[0]).  Errors are reported on
 * ctxs[0]: MCD_E_INVALID (bad arguments, more than 16 sites, contexts on
 * different devices), MCD_E_NODEVICE, MCD_E_STATE (no basis), MCD_E_OOM.
 *
 * mcd_batch_apply: y_i = H~_i x_i for every instance (App. B projection, as
 * mcd_apply), single column.  x, y: device arrays of sum_i N_i elements of
 * dtype, instance i at offset N_0 + ... + N_{i-1}; x and y must not overlap.
 * All instances run in one persistent launch per pass that pulls (instance,
 * work item) units from a device queue; the launch grid is chosen by timing
 * candidates on the first batch of a given size. */
int mcd_batch_apply(mcd_ctx* const* ctxs, int n_inst, const void* x, void* y, int dtype);
/* App. B Lanczos ground state of every instance, all instances advancing in
 * lockstep (one launch per phase for the batch; the launches of 16 steps are
 * captured once in a CUDA graph and replayed).  Each instance stops when its
 * residual estimate b_{m+1} |e_m^T y| < tol max(1, |E0|) or at max_iter
 * (1 <= max_iter <= 100000).  Start vectors as mcd_lanczos_ground with the
 * same seed.  All Krylov vectors are kept (MCD_E_OOM if they do not fit).
 * E0: host [n_inst]; iters, residual: host [n_inst] or NULL.  psi: NULL or
 * host [n_inst] of device pointers (each NULL or N_i elements of dtype) that
 * receive the normalised Ritz vectors.  The MCD_F32 form returns each
 * instance's fp64 Rayleigh quotient of its Ritz vector.  Status:
 * MCD_E_NOT_CONVERGED if some instance reached max_iter with tol > 0 (E0 is
 * still filled), MCD_E_BREAKDOWN on a non-finite coefficient. */
int mcd_batch_lanczos_ground(mcd_ctx* const* ctxs, int n_inst, int max_iter, double tol, uint64_t seed,
                             int dtype, double* E0, int* iters, double* residual, void* const* psi);

/* Lanczos coefficients of the last mcd_lanczos_ground: a[cap], b[cap]
 * (b[0] = 0); *m = number of steps. Host arrays. */
int mcd_lanczos_coeffs(const mcd_ctx* ctx, double* a, double* b, int cap, int* m);

/* Timing of H*v launches recorded with MCD_OPT_KERNEL_TIMING since the last
 * reset: total milliseconds and launch count per kernel class
 * (0 = dn-major up-hop pass, 1 = up-major dn-hop + diagonal pass,
 *  2 = Krylov update, 3 = plain kernel).  reset != 0 clears after reading. */
int mcd_kernel_times(mcd_ctx* ctx, double* ms, int64_t* count, int n_classes, int reset);

/* Connection cache of the current basis and Hamiltonian (MCD_OPT_HV_CACHE):
 * *bytes = device bytes of its records including padding, *n_conn = stored
 * hops (both passes; equals the off-diagonal nonzeros of H~), *rec_bytes =
 * bytes per record (2: items whose blocks hold at most 16383 states take
 * 2-byte records, larger ones 4; 4: every item), all 0 when no cache is
 * built; *wait_errors = 1 when a bounded wait inside a cached H*v kernel ran
 * out since the records were built (its results are then not to be used).
 * Any pointer may be NULL.  Synchronises the context's stream.  MCD_E_STATE
 * without a basis. */
int mcd_hv_cache_info(mcd_ctx* ctx, int64_t* bytes, int64_t* n_conn, int* rec_bytes, int* wait_errors);

/* Number of kernels this context has launched since creation (all entry
 * points); *n receives the count. */
int mcd_launch_count(const mcd_ctx* ctx, int64_t* n);

#ifdef __cplusplus
}
#endif
#endif /* MCD_H */
