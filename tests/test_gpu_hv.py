"""GPU parity of the H~ x path through the C ABI against the oracle:
connection lists and signs bit-exact, diagonal, y = H~ x within the rounding
bound of the arithmetic, for fp64 and fp32 vectors, one and many columns,
ragged widths, padded rows, both kernel variants and the edge cases (one
state, an oversized block, 32 sites, site-dependent eps and U)."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from oracle import fock, hamiltonian as H, sampler as S
from workloads import configs as C, lattice as L, random_block

from gpu_common import U32, U64, apply_bound, device_ctx, golden, model, row_terms_bound

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def n_bonds(t):
    return int(np.count_nonzero(np.triu(t, 1)))


def check_apply(ctx, P, t, ncols, dtype, ld=None, seed=0, offset=0):
    n = P.n
    ld = ncols if ld is None else ld
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    X = random_block(n, ncols, seed, dtype)
    Xfull = np.zeros((n, ld), dtype=dtype)
    Xfull[:, :ncols] = X
    # optional element offset to make the rows unaligned
    xbuf = torch.zeros(n * ld + offset, dtype=tdt, device=DEV)
    ybuf = torch.full((n * ld + offset,), float("nan"), dtype=tdt, device=DEV)
    xbuf[offset:] = torch.from_numpy(Xfull.reshape(-1)).to(DEV)
    x = xbuf[offset:].view(n, ld)
    y = ybuf[offset:].view(n, ld)
    st = ctx.L.mcd_apply(ctx.h, x.data_ptr(), y.data_ptr(), ncols, ld,
                         pkg.MCD_F64 if dtype == np.float64 else pkg.MCD_F32)
    ctx._check(st)
    torch.cuda.synchronize()
    Y = y.cpu().numpy()[:, :ncols].astype(np.float64)
    Xd = X.astype(np.float64)
    ref = P.sparse() @ Xd
    absHx = H.apply_abs(P, Xd)
    u = U64 if dtype == np.float64 else U32
    nt = row_terms_bound(n_bonds(t))
    # computed side within nt*u, reference (scipy fp64) within nt*U64
    bound = apply_bound(absHx, nt, u) + apply_bound(absHx, nt, U64)
    err = np.abs(Y - ref)
    assert np.all(err <= bound), (float(np.max(err)), float(np.max(err - bound)))
    if ld > ncols:   # padding untouched
        assert np.all(np.isnan(y.cpu().numpy()[:, ncols:]))
    return float(np.max(err))


@pytest.fixture(scope="module")
def ring8():
    w = C.ring8_u4()
    ctx = device_ctx(w)
    B = ctx.mcd_get_basis()
    P = H.build(model(w), B)
    return w, ctx, B, P


@pytest.fixture(scope="module")
def tilted12():
    w = C.tilted12_u8()
    ctx = device_ctx(w)
    B = ctx.mcd_get_basis()
    P = H.build(model(w), B)
    return w, ctx, B, P


def test_basis_matches_oracle_sampler(ring8, tilted12):
    for w, ctx, B, P in (ring8, tilted12):
        ref = S.sample_basis(w.n_sites, w.lat.t, w.U_sites, w.n_up, w.n_dn, w.n_f, w.beta,
                             [w.seed_word()], seed=w.seed)
        assert np.array_equal(B, ref)


@pytest.mark.parametrize("which", ["ring8", "tilted12"])
def test_connections_bit_exact(which, request):
    w, ctx, B, P = request.getfixturevalue(which)
    nnz = ctx.mcd_connections()
    assert nnz == P.nnz_offdiag() == golden()[f"{which}_mc_nnz"]
    rows = torch.empty(nnz, dtype=torch.int64, device=DEV)
    cols = torch.empty(nnz, dtype=torch.int64, device=DEV)
    vals = torch.empty(nnz, dtype=torch.float64, device=DEV)
    assert ctx.mcd_connections(rows, cols, vals) == nnz
    r, c, v = rows.cpu().numpy(), cols.cpu().numpy(), vals.cpu().numpy()
    o = np.lexsort((c, r))
    assert np.array_equal(r[o], P.rows) and np.array_equal(c[o], P.cols)
    assert np.array_equal(v[o], P.vals)          # t_ij * sign: exact
    info = ctx.mcd_basis_info()
    assert info["nnz_offdiag"] == nnz and info["n_states"] == len(B)
    up, dn = fock.split(B, w.n_sites)
    assert info["n_up_blocks"] == len(np.unique(up)) and info["n_dn_blocks"] == len(np.unique(dn))


@pytest.mark.parametrize("which", ["ring8", "tilted12"])
def test_diagonal(which, request):
    w, ctx, B, P = request.getfixturevalue(which)
    d = torch.empty(len(B), dtype=torch.float64, device=DEV)
    ctx.mcd_diagonal(d)
    assert np.array_equal(d.cpu().numpy(), P.diag)   # integer-valued here: exact


# (algorithm, states per hash work item, connection cache): the cached path
# (records built by the first H~x, then streamed), the matrix-free default
# kernels (bitmap for <= 16 sites, hash above), the in-block binary search,
# and the hash kernel at its default item size (1024) and at 64 states per
# item, where most blocks are split into chunks that share a table in device
# memory
ALGOS = [(pkg.HV_AUTO, 1024, pkg.CACHE_REQUIRED), (pkg.HV_AUTO, 1024, pkg.CACHE_OFF),
         (pkg.HV_SEARCH, 1024, pkg.CACHE_OFF), (pkg.HV_HASH, 1024, pkg.CACHE_OFF),
         (pkg.HV_HASH, 64, pkg.CACHE_OFF)]
ALGO_IDS = ["cached", "matrix-free", "search", "hash", "hash-item64"]


@pytest.fixture(params=ALGOS, ids=ALGO_IDS)
def algo(request):
    return request.param


def with_algo(ctx, algo):
    a, item = algo[:2]
    ctx.mcd_set_option(pkg.MCD_OPT_HV_ALGO, a)
    ctx.mcd_set_option(pkg.MCD_OPT_HASH_ITEM, item)
    ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, algo[2] if len(algo) > 2 else pkg.CACHE_AUTO)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("ncols", [1, 3, 8, 24, 48])
def test_apply_ring8(ring8, dtype, ncols, algo):
    w, ctx, B, P = ring8
    with_algo(ctx, algo)
    check_apply(ctx, P, w.lat.t, ncols, dtype, seed=ncols)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("ncols,ld,offset", [(1, 1, 0), (12, 12, 0), (24, 24, 0), (5, 8, 0),
                                             (4, 4, 1), (130, 132, 0)])
def test_apply_tilted12(tilted12, dtype, ncols, ld, offset, algo):
    w, ctx, B, P = tilted12
    with_algo(ctx, algo)
    check_apply(ctx, P, w.lat.t, ncols, dtype, ld=ld, offset=offset, seed=7 + ncols)


def test_apply_exact_rows_fsum(ring8):
    # against correctly rounded rows (math.fsum) on the small case
    w, ctx, B, P = ring8
    X = random_block(len(B), 2, 3, np.float64)
    x = torch.from_numpy(X).to(DEV)
    y = torch.empty_like(x)
    ctx.mcd_apply(x, y)
    torch.cuda.synchronize()
    ref = H.apply_exact(P, X)
    bound = apply_bound(H.apply_abs(P, X), row_terms_bound(n_bonds(w.lat.t)), U64)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= bound)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_plain_kernel_variant(tilted12, dtype):
    w, ctx, B, P = tilted12
    with_algo(ctx, (pkg.HV_PLAIN, 1024))
    try:
        check_apply(ctx, P, w.lat.t, 2, dtype, seed=99)
    finally:
        with_algo(ctx, (pkg.HV_AUTO, 1024))


def test_single_state_basis(algo):
    w = C.ring8_u4()
    ctx = device_ctx(w, basis=np.array([w.seed_word()], dtype=np.uint64))
    with_algo(ctx, algo)
    P = H.build(model(w), np.array([w.seed_word()], dtype=np.uint64))
    check_apply(ctx, P, w.lat.t, 3, np.float64)


def test_tiny_lattice_small_bitmap(algo):
    # 3 sites: the bitmap has fewer than 32 bits
    lat = L.ring(3)
    w = C.Workload("ring3", lat, 2.0, 1, 2, 0, 0.5)
    B = fock.sector(3, 1, 2)
    ctx = device_ctx(w, basis=B)
    with_algo(ctx, algo)
    P = H.build(model(w), B)
    for dt in (np.float64, np.float32):
        check_apply(ctx, P, lat.t, 1, dt)
        check_apply(ctx, P, lat.t, 2, dt)


def test_oversized_block_uses_global_search():
    # one up word with all C(16, 8) = 12870 down words: a block larger than
    # the shared-memory staging area of a CTA
    lat = L.ring(16)
    w = C.Workload("ring16", lat, 8.0, 8, 8, 0, 0.2)
    ups = fock.words_with_popcount(16, 8)
    dns = np.array(fock.words_with_popcount(16, 8), dtype=np.uint64)
    big = (np.uint64(ups[100]) << np.uint64(16)) | dns
    rng = np.random.default_rng(4)
    others = [(np.uint64(ups[k]) << np.uint64(16)) | dns[rng.choice(len(dns), 300, replace=False)]
              for k in (3, 99, 101, 2000)]
    B = np.unique(np.concatenate([big] + others))
    ctx = device_ctx(w, basis=B)
    P = H.build(model(w), B)
    for algo in ALGOS:
        with_algo(ctx, algo)
        for dt in (np.float64, np.float32):
            check_apply(ctx, P, lat.t, 1, dt)
            check_apply(ctx, P, lat.t, 6, dt)
            check_apply(ctx, P, lat.t, 33, dt)


def test_thirty_two_sites_random_hoppings_and_site_terms():
    # 32 sites (words use all 64 bits), random long-range t_ij, site-dependent
    # eps_i and U_i (non-uniform diagonal path)
    n = 32
    rng = np.random.default_rng(8)
    t = np.zeros((n, n))
    for _ in range(60):
        i, j = rng.choice(n, 2, replace=False)
        t[i, j] = t[j, i] = rng.normal()
    lat = L.Lattice("rand32", n, t, np.zeros((n, 2), int), np.arange(n) % 2)
    eps = rng.normal(size=n)
    U = rng.uniform(0, 8, size=n)
    w = C.Workload("rand32", lat, 0.0, 3, 2, 0, 0.5)
    seed = (np.uint64(0b111 << 29) << np.uint64(32)) | np.uint64(0b11)
    B = S.sample_basis(n, t, U, 3, 2, 20000, 0.5, [int(seed)], seed=1)
    import paper_2509_22975_gb300 as pk
    ctx = pk.Context(0)
    ctx.mcd_set_hamiltonian(t, eps, U, 3, 2)
    ctx.mcd_set_basis(B)
    P = H.build(H.Model(n, t, eps, U), B)
    d = torch.empty(len(B), dtype=torch.float64, device=DEV)
    ctx.mcd_diagonal(d)
    assert np.max(np.abs(d.cpu().numpy() - P.diag)) <= 4 * n * U64 * np.max(np.abs(P.diag))
    nnz = ctx.mcd_connections()
    assert nnz == P.nnz_offdiag()
    for algo in ALGOS:
        with_algo(ctx, algo)
        for dt in (np.float64, np.float32):
            check_apply(ctx, P, t, 1, dt, seed=2)
            check_apply(ctx, P, t, 8, dt, seed=3)


@pytest.fixture(scope="module")
def rect24():
    # 6x4 t-t' cluster (24 sites, 11 + 11 electrons): a 60,000-state MC basis
    w = C.rect24_u8()
    ctx = device_ctx(w, nf=60000)
    B = ctx.mcd_get_basis()
    P = H.build(model(w), B)
    return w, ctx, B, P


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("ncols,ld,offset", [(1, 1, 0), (3, 3, 0), (24, 24, 0), (48, 48, 0), (5, 8, 0),
                                             (4, 4, 1), (70, 72, 0)])
def test_apply_rect24(rect24, dtype, ncols, ld, offset, algo):
    # more than 16 sites: the default path is the hash kernel
    w, ctx, B, P = rect24
    with_algo(ctx, algo)
    check_apply(ctx, P, w.lat.t, ncols, dtype, ld=ld, offset=offset, seed=11 + ncols)


def test_rect24_item_sizes(rect24):
    # every item size gives the same y (lookups are exact), fp64 bit for bit
    # across item sizes and against the binary-search kernel
    w, ctx, B, P = rect24
    x = torch.from_numpy(random_block(len(B), 2, 5, np.float64)).to(DEV)
    ys = []
    for algo in [(pkg.HV_SEARCH, 1024)] + [(pkg.HV_HASH, k) for k in (64, 128, 512, 1024, 4096)]:
        with_algo(ctx, algo)
        y = torch.empty_like(x)
        ctx.mcd_apply(x, y)
        ys.append(y.cpu().numpy())
    with_algo(ctx, (pkg.HV_AUTO, 1024))
    ref = P.sparse() @ x.cpu().numpy()
    bound = apply_bound(H.apply_abs(P, x.cpu().numpy()), row_terms_bound(n_bonds(w.lat.t)), 2 * U64)
    for y in ys:
        assert np.all(np.abs(y - ref) <= bound)
    for y in ys[2:]:
        assert np.array_equal(y, ys[1])


def test_block_above_table_limit_uses_search():
    # 20 sites: one up word with all C(20, 10) = 184,756 down words, a block
    # too large for 16-bit table positions (binary search inside the hash
    # kernel), plus small blocks
    n = 20
    lat = L.ring(n)
    w = C.Workload("ring20", lat, 4.0, 10, 10, 0, 0.4)
    dns = np.array(fock.words_with_popcount(n, 10), dtype=np.uint64)
    ups = fock.words_with_popcount(n, 10)
    rng = np.random.default_rng(6)
    parts = [(np.uint64(ups[500]) << np.uint64(n)) | dns]
    parts += [(np.uint64(ups[k]) << np.uint64(n)) | dns[rng.choice(len(dns), 2000, replace=False)]
              for k in (1, 499, 501, 7000)]
    B = np.unique(np.concatenate(parts))
    ctx = device_ctx(w, basis=B)
    P = H.build(model(w), B)
    for algo in [(pkg.HV_AUTO, 1024), (pkg.HV_HASH, 256)]:
        with_algo(ctx, algo)
        for dt in (np.float64, np.float32):
            check_apply(ctx, P, lat.t, 1, dt, seed=4)
            check_apply(ctx, P, lat.t, 6, dt, seed=5)


def test_hash_item_option_errors(ring8):
    w, ctx, B, P = ring8
    for bad in (0, 32, 100, 8192):
        with pytest.raises(pkg.MCDError):
            ctx.mcd_set_option(pkg.MCD_OPT_HASH_ITEM, bad)
    with pytest.raises(pkg.MCDError):
        ctx.mcd_set_option(pkg.MCD_OPT_HV_ALGO, 4)


def test_argument_errors(ring8):
    w, ctx, B, P = ring8
    x = torch.zeros(len(B), dtype=torch.float64, device=DEV)
    for args, code in [((x.data_ptr(), x.data_ptr(), 1, 1, 0), -1),           # aliasing
                       ((x.data_ptr(), x.data_ptr() + 8 * len(B), 0, 1, 0), -1),   # ncols 0
                       ((x.data_ptr(), x.data_ptr() + 8 * len(B), 2, 1, 0), -1),   # ld < ncols
                       ((x.data_ptr(), x.data_ptr() + 8 * len(B), 1, 1, 7), -1)]:  # dtype
        assert ctx.L.mcd_apply(ctx.h, *args) == code


def test_multi_column_list_overflow():
    # complete bipartite K(8,8), uniform t (8 partner classes): the down word
    # with all electrons on one side has 64 active bonds, every target in the
    # basis (one up word with all C(16, 8) down words), more hops than a
    # state's list in the multi-column kernel holds; they are found again
    n = 16
    t = np.zeros((n, n))
    for i in range(8):
        for j in range(8, 16):
            t[i, j] = t[j, i] = -1.0
    lat = L.Lattice("k88", n, t, np.zeros((n, 2), int), np.arange(n) // 8)
    w = C.Workload("k88", lat, 2.0, 8, 8, 0, 0.2)
    dns = np.array(fock.words_with_popcount(n, 8), dtype=np.uint64)
    ups = fock.words_with_popcount(n, 8)
    rng = np.random.default_rng(9)
    B = np.unique(np.concatenate([(np.uint64(0x00FF) << np.uint64(n)) | dns] +
                                 [(np.uint64(ups[k]) << np.uint64(n)) | dns[rng.choice(len(dns), 500, replace=False)]
                                  for k in (5, 700, 9000)]))
    ctx = device_ctx(w, basis=B)
    P = H.build(model(w), B)
    for algo in [(pkg.HV_AUTO, 1024), (pkg.HV_SEARCH, 1024)]:
        with_algo(ctx, algo)
        for dt in (np.float64, np.float32):
            for nc in (2, 8, 24):
                check_apply(ctx, P, t, nc, dt, seed=nc)
