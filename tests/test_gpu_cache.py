"""Connection cache of H~x (MCD_OPT_HV_CACHE) through the C ABI: the stored
hops are the oracle's off-diagonal nonzeros (count, record width), y = H~x
from the records within the rounding bound of the oracle for one and many
columns, fp64 and fp32, both record widths (2-byte records with <= 2
amplitudes, 4-byte ones with amplitude classes or per-bond coefficients),
rebuilt after a new Hamiltonian or basis, released when switched off;
Lanczos E0 from the cached path against the matrix-free one; determinism;
the band-Lanczos Green function with and without the cache."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from oracle import fock, hamiltonian as H, sampler as S
from workloads import configs as C, lattice as L, random_block

from gpu_common import U32, U64, apply_bound, device_ctx, model, row_terms_bound

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def n_bonds(t):
    return int(np.count_nonzero(np.triu(t, 1)))


def apply(ctx, X):
    x = torch.from_numpy(np.ascontiguousarray(X)).to(DEV)
    y = torch.full_like(x, float("nan"))
    ctx.mcd_apply(x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def check(ctx, P, t, ncols, dtype, seed=0):
    X = random_block(P.n, ncols, seed, dtype)
    if ncols == 1:
        X = X[:, 0].copy()
    Y = apply(ctx, X)
    Xd = X.astype(np.float64)
    ref = P.sparse() @ Xd
    absHx = H.apply_abs(P, Xd)
    u = U64 if dtype == np.float64 else U32
    nt = row_terms_bound(n_bonds(t))
    bound = apply_bound(absHx, nt, u) + apply_bound(absHx, nt, U64)
    assert np.all(np.abs(Y - ref) <= bound), float(np.max(np.abs(Y - ref) - bound))


def cached_ctx(w, B, t=None, eps=None, U=None):
    ctx = pkg.Context(0)
    ctx.mcd_set_hamiltonian(w.lat.t if t is None else t, w.eps if eps is None else eps,
                            w.U if U is None else U, w.n_up, w.n_dn)
    ctx.mcd_set_basis(B)
    ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_REQUIRED)
    return ctx


@pytest.mark.parametrize("name,nf", [("ring8_u4", 2000), ("tilted12_u8", 1 << 16), ("square16_u8", 200000),
                                     ("rect24_u8", 60000)])
def test_records_are_the_nonzeros(name, nf):
    w = getattr(C, name)()
    B = S.sample_basis(w.n_sites, w.lat.t, w.U_sites, w.n_up, w.n_dn, nf, w.beta, [w.seed_word()], seed=w.seed) \
        if nf <= 2000 else None
    ctx = device_ctx(w, basis=B, nf=nf)
    B = ctx.mcd_get_basis()
    ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_REQUIRED)
    assert ctx.mcd_hv_cache_info()["bytes"] == 0          # built by the first H~x
    P = H.build(model(w), B)
    for dt in (np.float64, np.float32):
        for nc in (1, 8, 24):
            check(ctx, P, w.lat.t, nc, dt, seed=nc)
    info = ctx.mcd_hv_cache_info()
    assert info["n_conn"] == P.nnz_offdiag() and info["wait_errors"] == 0
    amps = np.unique(np.round(w.lat.t[np.triu(w.lat.t, 1) != 0], 12))
    assert info["rec_bytes"] == (2 if len(amps) <= 2 else 4)
    # padding: at least the records, 256-byte groups
    assert info["bytes"] >= info["n_conn"] * info["rec_bytes"] and info["bytes"] % 256 == 0


def test_four_byte_records_amplitude_classes_and_bonds():
    # 12 sites with 3 distinct amplitudes (classes) and with 30 distinct ones
    # (no class table: one coefficient per bond)
    w = C.tilted12_u8()
    B = S.sample_basis(12, w.lat.t, w.U_sites, 6, 6, 30000, w.beta, [w.seed_word()], seed=3)
    rng = np.random.default_rng(5)
    iu = np.argwhere(np.triu(w.lat.t, 1) != 0)
    for kind in ("classes", "bonds"):
        t = w.lat.t.copy()
        for r, (i, j) in enumerate(iu):
            v = [-1.0, -0.5, 0.25][r % 3] if kind == "classes" else rng.normal()
            t[i, j] = t[j, i] = v
        for i, j in [(0, 5), (2, 9)]:        # longer-range bonds
            t[i, j] = t[j, i] = 0.3 if kind == "classes" else rng.normal()
        eps = rng.normal(size=12) * (kind == "bonds")
        U = np.full(12, 6.0) if kind == "classes" else rng.uniform(2, 8, 12)
        ctx = cached_ctx(w, B, t=t, eps=eps, U=U)
        P = H.build(H.Model(12, t, eps, U), B)
        for dt in (np.float64, np.float32):
            for nc in (1, 5, 24):
                check(ctx, P, t, nc, dt, seed=nc)
        info = ctx.mcd_hv_cache_info()
        assert info["rec_bytes"] == 4 and info["n_conn"] == P.nnz_offdiag()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_unaligned_single_column(dtype):
    # x and y one element past a 16-byte boundary: the streaming kernel cannot
    # copy rows of x in 16-byte units and reads them from global memory
    w = C.square16_u8()
    ctx = device_ctx(w, nf=60000)
    ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_REQUIRED)
    B = ctx.mcd_get_basis()
    P = H.build(model(w), B)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    X = random_block(len(B), 1, 5, dtype)[:, 0].copy()
    for off in (0, 1, 3):
        xb = torch.zeros(len(B) + 4, dtype=tdt, device=DEV)
        yb = torch.full((len(B) + 4,), float("nan"), dtype=tdt, device=DEV)
        xb[off:off + len(B)] = torch.from_numpy(X).to(DEV)
        ctx.mcd_apply(xb[off:off + len(B)], yb[off:off + len(B)])
        torch.cuda.synchronize()
        Y = yb[off:off + len(B)].cpu().numpy().astype(np.float64)
        ref = P.sparse() @ X.astype(np.float64)
        u = U64 if dtype == np.float64 else U32
        nt = row_terms_bound(n_bonds(w.lat.t))
        absHx = H.apply_abs(P, X.astype(np.float64))
        assert np.all(np.abs(Y - ref) <= apply_bound(absHx, nt, u) + apply_bound(absHx, nt, U64))
        assert torch.isnan(yb[:off]).all() and torch.isnan(yb[off + len(B):]).all()
    assert ctx.mcd_hv_cache_info()["wait_errors"] == 0


def test_rebuilt_for_new_hamiltonian_and_basis_and_released():
    w = C.tilted12_u8()
    ctx = device_ctx(w, nf=20000)
    B = ctx.mcd_get_basis()
    ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_REQUIRED)
    check(ctx, H.build(model(w), B), w.lat.t, 1, np.float64)
    assert ctx.mcd_hv_cache_info()["n_conn"] > 0
    # new amplitudes, same bonds: records hold the old classes until rebuilt
    t2 = 0.7 * w.lat.t
    ctx.mcd_set_hamiltonian(t2, w.eps, w.U, w.n_up, w.n_dn)
    assert ctx.mcd_hv_cache_info()["bytes"] == 0
    check(ctx, H.build(H.Model(12, t2, w.eps, w.U_sites), B), t2, 3, np.float64)
    # a smaller basis in the same sector
    B2 = B[::3].copy()
    ctx.mcd_set_basis(B2)
    assert ctx.mcd_hv_cache_info()["bytes"] == 0
    P2 = H.build(H.Model(12, t2, w.eps, w.U_sites), B2)
    check(ctx, P2, t2, 1, np.float32)
    assert ctx.mcd_hv_cache_info()["n_conn"] == P2.nnz_offdiag()
    ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_OFF)
    assert ctx.mcd_hv_cache_info()["bytes"] == 0
    check(ctx, P2, t2, 1, np.float32)
    assert ctx.mcd_hv_cache_info()["bytes"] == 0
    with pytest.raises(pkg.MCDError):
        ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, 3)


@pytest.mark.parametrize("name,nf", [("square16_u8", 300000), ("rect24_u8", 200000)])
def test_lanczos_cached_equals_matrix_free(name, nf):
    w = getattr(C, name)()
    res = {}
    for mode in (pkg.CACHE_OFF, pkg.CACHE_REQUIRED):
        ctx = device_ctx(w, nf=nf)
        ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, mode)
        r64 = ctx.mcd_lanczos_ground(1000, 1e-11, 0, pkg.MCD_F64, allow_not_converged=True)
        r32 = ctx.mcd_lanczos_ground(600, 1e-9, 0, pkg.MCD_F32, allow_not_converged=True)
        res[mode] = (r64["E0"], r32["E0"])
    e_off, e_on = res[pkg.CACHE_OFF], res[pkg.CACHE_REQUIRED]
    assert abs(e_on[0] - e_off[0]) <= 1e-9 * abs(e_off[0])
    assert abs(e_on[1] - e_off[0]) < 1e-6


def test_deterministic_and_ragged_columns():
    w = C.square16_u8()
    ctx = device_ctx(w, nf=100000)
    ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_REQUIRED)
    B = ctx.mcd_get_basis()
    P = H.build(model(w), B)
    X = random_block(len(B), 1, 2, np.float32)[:, 0].copy()
    assert np.array_equal(apply(ctx, X), apply(ctx, X))
    for nc in (2, 3, 7, 12, 13, 33, 48, 64):
        check(ctx, P, w.lat.t, nc, np.float32, seed=nc)
    for nc in (2, 9, 31):
        check(ctx, P, w.lat.t, nc, np.float64, seed=nc)


def test_band_green_with_and_without_cache():
    # few block steps (the Krylov vectors of both runs stay orthogonal to
    # rounding level, so the two G agree to rounding; after many steps the
    # unconverged low-frequency poles move with any change of rounding)
    w = C.tilted12_u8()
    orb = [(i, 0) for i in range(4)]
    z = 1j * (2 * np.arange(4) + 1) * np.pi / 20.0
    out = []
    for mode in (pkg.CACHE_OFF, pkg.CACHE_REQUIRED):
        ctx = device_ctx(w, nf=30000)
        ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, mode)
        n = ctx.mcd_basis_info(nnz=False)["n_states"]
        psi = torch.empty(n, dtype=torch.float64, device=DEV)
        ctx.mcd_lanczos_ground(1000, 1e-13, 0, pkg.MCD_F64, psi=psi)
        G, dp, dm = ctx.mcd_band_lanczos_green(orb, 10, 1.0, z)
        out.append((G, dp, dm))
    # at w_t = 1 the excited spaces take every ground-state component above
    # zero: the two kernels' rounding can leave a few symmetry-zero components
    # at noise level in one run and not the other (weights ~1e-30, nothing in G)
    assert abs(out[0][1] - out[1][1]) <= 1e-4 * out[0][1] and abs(out[0][2] - out[1][2]) <= 1e-4 * out[0][2]
    assert np.max(np.abs(out[0][0] - out[1][0])) < 1e-9 * max(1.0, np.max(np.abs(out[0][0])))


def test_set_basis_from_pinned_tensor_and_device_checks():
    # host words go straight to the device and are checked there: a pinned
    # torch tensor gives the same basis and products as a numpy array;
    # unsorted words and words outside the sector are refused with the same
    # codes as on a host-only context, and the context stays usable
    w = C.tilted12_u8()
    ctx = device_ctx(w, nf=5000)
    B = ctx.mcd_get_basis()
    P = H.build(model(w), B)
    t = torch.from_numpy(B.view(np.int64)).pin_memory()
    ctx.mcd_set_basis(t)
    assert np.array_equal(ctx.mcd_get_basis(), B)
    check(ctx, P, w.lat.t, 1, np.float64)
    bad = B.copy()
    bad[[10, 11]] = bad[[11, 10]]
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_set_basis(bad)
    assert e.value.status == -1
    up = (1 << 12) - 1                       # 12 up electrons: outside the 6 + 6 sector
    outside = np.sort(np.concatenate([B[:100], np.array([(up << 12) | 0b111111], dtype=np.uint64)]))
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_set_basis(np.unique(outside))
    assert e.value.status == -2
    ctx.mcd_set_basis(B)
    check(ctx, P, w.lat.t, 3, np.float32)


@pytest.mark.parametrize("cut", [1, 2, 3, 5])
def test_single_column_basis_size_not_a_multiple_of_four(cut):
    # the dn-major copy of x before pass B moves four positions per thread;
    # the last n mod 4 positions take the scalar tail
    w = C.square16_u8()
    ctx = device_ctx(w, nf=40000)
    B = ctx.mcd_get_basis()[:-cut]
    P = H.build(model(w), B)
    ctx = cached_ctx(w, B)
    for dtype in (np.float32, np.float64):
        check(ctx, P, w.lat.t, 1, dtype, seed=cut)
    info = ctx.mcd_hv_cache_info()
    assert info["n_conn"] == P.nnz_offdiag() and info["wait_errors"] == 0


@pytest.mark.parametrize("name,nf", [("tilted12_u8", 1 << 16), ("square16_u8", 200000), ("rect24_u8", 60000)])
def test_both_many_column_kernels_and_the_timed_pick(name, nf):
    # the pipelined-tile kernel and the CTA-per-item kernel, each forced,
    # against the oracle for 2, 8, 24 and 48 columns in fp32 and fp64; the
    # timed pick (default) gives bit for bit what the kernel it keeps gives
    w = getattr(C, name)()
    ctx = device_ctx(w, nf=nf)
    ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_REQUIRED)
    B = ctx.mcd_get_basis()
    P = H.build(model(w), B)
    for mode in (pkg.HV_COLS_TILES, pkg.HV_COLS_ITEMS):
        ctx.mcd_set_option(pkg.MCD_OPT_HV_COLS, mode)
        for dt in (np.float64, np.float32):
            for nc in (2, 8, 24, 48):
                check(ctx, P, w.lat.t, nc, dt, seed=nc + mode)
    X = random_block(len(B), 24, 7, np.float32)
    ys = {}
    for mode in (pkg.HV_COLS_AUTO, pkg.HV_COLS_TILES, pkg.HV_COLS_ITEMS):
        ctx.mcd_set_option(pkg.MCD_OPT_HV_COLS, mode)
        ys[mode] = [apply(ctx, X) for _ in range(2)]   # auto: the first call times both, the second uses the pick
    assert np.array_equal(ys[pkg.HV_COLS_TILES][0], ys[pkg.HV_COLS_TILES][1])
    assert np.array_equal(ys[pkg.HV_COLS_ITEMS][0], ys[pkg.HV_COLS_ITEMS][1])
    picked = ys[pkg.HV_COLS_AUTO][1]
    assert np.array_equal(picked, ys[pkg.HV_COLS_TILES][0]) or np.array_equal(picked, ys[pkg.HV_COLS_ITEMS][0])
