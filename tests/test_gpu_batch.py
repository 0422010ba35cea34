"""Batches of impurity models (2x2 plaquette + 8 bath sites, uneven Monte
Carlo bases) through the C ABI: batched H~v equal to each instance's own
mcd_apply bit for bit and to the oracle within the rounding bound; batched
Lanczos E0 against the single-instance solver and against scipy's Lanczos on
the oracle's H~; fp32 against fp64; Ritz vectors; determinism; errors; and
the 256-instance batch at full size."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from oracle import hamiltonian as H
from workloads import impurity as IM

from gpu_common import U32, U64, apply_bound, row_terms_bound

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def make_ctx(m, nf=None):
    ctx = pkg.Context(0)
    ctx.mcd_set_hamiltonian(m.t, m.eps, m.U_sites, m.n_up, m.n_dn)
    ctx.mcd_build_basis(m.seed, nf or m.n_f, m.beta, [m.seed_word()])
    return ctx


def model(m):
    return H.Model(m.n_sites, m.t, m.eps, m.U_sites)


@pytest.fixture(scope="module")
def batch12():
    ms = IM.batch(12)
    ms[0].n_f, ms[1].n_f = 1000, 900      # small ones the oracle solves densely
    ctxs = [make_ctx(m) for m in ms]
    return ms, ctxs


def concat(parts, dtype):
    return torch.cat([torch.as_tensor(p, dtype=dtype) for p in parts]).to(DEV)


@pytest.mark.parametrize("split", [0, 1, 2, 4])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_apply_equals_single_and_oracle(batch12, dtype, split):
    # every work-unit size (timed pick, or 1024, 512 and 256 states per
    # unit) gives the same product bit for bit
    ms, ctxs = batch12
    sizes = [c.mcd_basis_info(nnz=False)["n_states"] for c in ctxs]
    g = torch.Generator(device=DEV).manual_seed(3)
    x = torch.randn(sum(sizes), dtype=dtype, device=DEV, generator=g)
    y = torch.full_like(x, float("nan"))
    ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_SPLIT, split)
    try:
        pkg.mcd_batch_apply(ctxs, x, y)
    finally:
        ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_SPLIT, 0)
    torch.cuda.synchronize()
    off = np.concatenate([[0], np.cumsum(sizes)])
    u = U64 if dtype == torch.float64 else U32
    for i, (m, c) in enumerate(zip(ms, ctxs)):
        xi = x[off[i]:off[i + 1]].clone()
        yi = torch.empty_like(xi)
        c.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_OFF)   # the matrix-free kernel the batch shares
        c.mcd_apply(xi, yi)
        c.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_AUTO)
        torch.cuda.synchronize()
        assert torch.equal(yi, y[off[i]:off[i + 1]])          # same kernel arithmetic
        if i < 4:
            P = H.build(model(m), c.mcd_get_basis())
            X = xi.double().cpu().numpy()
            ref = P.sparse() @ X
            nt = row_terms_bound(int(np.count_nonzero(np.triu(m.t, 1))))
            absHx = H.apply_abs(P, X)
            bound = apply_bound(absHx, nt, u) + apply_bound(absHx, nt, U64)
            assert np.all(np.abs(yi.double().cpu().numpy() - ref) <= bound)


@pytest.fixture(params=[pkg.BATCH_POOL, pkg.BATCH_LOCKSTEP], ids=["pool", "lockstep"])
def mode(request, batch12):
    # both forms of the batched Lanczos (MCD_OPT_BATCH_MODE, read from the first context)
    batch12[1][0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, request.param)
    yield request.param
    batch12[1][0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_POOL)


def test_batch_lanczos_fp64_against_single_and_oracle(batch12, mode):
    import scipy.sparse.linalg as sla
    ms, ctxs = batch12
    r = pkg.mcd_batch_lanczos_ground(ctxs, 600, 1e-12, 0, pkg.MCD_F64)
    for i, (m, c) in enumerate(zip(ms, ctxs)):
        s = c.mcd_lanczos_ground(600, 1e-12, 0, pkg.MCD_F64)
        assert abs(r["E0"][i] - s["E0"]) <= 1e-10 * abs(s["E0"])
        if i < 2:
            P = H.build(model(m), c.mcd_get_basis())
            E_ref = float(np.linalg.eigvalsh(P.dense())[0])
        elif i < 5:
            P = H.build(model(m), c.mcd_get_basis())
            E_ref = float(sla.eigsh(P.sparse(), k=1, which="SA", tol=1e-14)[0][0])
        else:
            continue
        assert abs(r["E0"][i] - E_ref) <= 1e-10 * abs(E_ref)


def test_batch_lanczos_fp32_and_ritz_vectors(batch12, mode):
    ms, ctxs = batch12
    sizes = [c.mcd_basis_info(nnz=False)["n_states"] for c in ctxs]
    psi = [torch.empty(n, dtype=torch.float32, device=DEV) for n in sizes]
    r64 = pkg.mcd_batch_lanczos_ground(ctxs, 600, 1e-12, 0, pkg.MCD_F64)
    r32 = pkg.mcd_batch_lanczos_ground(ctxs, 600, 1e-8, 0, pkg.MCD_F32, psi=psi, allow_not_converged=True)
    assert np.max(np.abs(r32["E0"] - r64["E0"])) < 1e-6
    for i in (0, 3, 7):
        p = psi[i].double()
        assert abs(float(p @ p) - 1.0) < 1e-5
        P = H.build(model(ms[i]), ctxs[i].mcd_get_basis())
        v = p.cpu().numpy()
        res = P.sparse() @ v - r32["E0"][i] * v
        assert np.linalg.norm(res) < 1e-3


@pytest.mark.parametrize("split", [1, 4])
def test_batch_lanczos_every_work_unit_size(batch12, split):
    # lockstep form: the fused <v, Hv> partials are summed per work unit:
    # another unit size sums them in another order, so E0 agrees within rounding
    ms, ctxs = batch12
    ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_LOCKSTEP)
    try:
        ref = pkg.mcd_batch_lanczos_ground(ctxs, 400, 1e-12, 0, pkg.MCD_F64)
        ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_SPLIT, split)
        r = pkg.mcd_batch_lanczos_ground(ctxs, 400, 1e-12, 0, pkg.MCD_F64)
    finally:
        ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_SPLIT, 0)
        ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_POOL)
    assert np.max(np.abs(r["E0"] - ref["E0"]) / np.abs(ref["E0"])) <= 1e-10


def test_batch_stream_pool_equals_separate_solves(batch12):
    # the default form: every instance's own (cached) solve on a stream pool
    # gives what separate mcd_lanczos_ground calls give, bit for bit
    ms, ctxs = batch12
    sizes = [c.mcd_basis_info(nnz=False)["n_states"] for c in ctxs]
    psi = [torch.empty(n, dtype=torch.float32, device=DEV) for n in sizes]
    r = pkg.mcd_batch_lanczos_ground(ctxs, 400, 1e-8, 0, pkg.MCD_F32, psi=psi, allow_not_converged=True)
    for i, c in enumerate(ctxs):
        p1 = torch.empty_like(psi[i])
        s = c.mcd_lanczos_ground(400, 1e-8, 0, pkg.MCD_F32, psi=p1, allow_not_converged=True)
        assert r["E0"][i] == s["E0"] and r["iters"][i] == s["iters"]
        assert torch.equal(p1, psi[i])
    ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_LOCKSTEP)
    try:
        ref = pkg.mcd_batch_lanczos_ground(ctxs, 400, 1e-8, 0, pkg.MCD_F32, allow_not_converged=True)
    finally:
        ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_POOL)
    assert np.max(np.abs(r["E0"] - ref["E0"])) < 1e-6


def test_batch_is_deterministic(batch12, mode):
    ms, ctxs = batch12
    a = pkg.mcd_batch_lanczos_ground(ctxs, 100, 0.0, 4, pkg.MCD_F32)
    b = pkg.mcd_batch_lanczos_ground(ctxs, 100, 0.0, 4, pkg.MCD_F32)
    assert np.array_equal(a["E0"], b["E0"]) and np.array_equal(a["iters"], b["iters"])


def test_batch_errors(batch12):
    ms, ctxs = batch12
    ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_LOCKSTEP)   # instances of one site count
    from workloads import configs as C
    w = C.rect24_u8()
    big = pkg.Context(0)
    big.mcd_set_hamiltonian(w.lat.t, w.eps, w.U, w.n_up, w.n_dn)
    big.mcd_build_basis(0, 1000, w.beta, [w.seed_word()])
    with pytest.raises(pkg.MCDError) as e:
        pkg.mcd_batch_lanczos_ground([ctxs[0], big], 50, 1e-10, 0, pkg.MCD_F64)
    assert e.value.status == -1
    nob = pkg.Context(0)
    nob.mcd_set_hamiltonian(ms[0].t, ms[0].eps, ms[0].U_sites, 6, 6)
    with pytest.raises(pkg.MCDError) as e:
        pkg.mcd_batch_lanczos_ground([ctxs[0], nob], 50, 1e-10, 0, pkg.MCD_F64)
    assert e.value.status == -8
    with pytest.raises(pkg.MCDError):
        pkg.mcd_batch_lanczos_ground(ctxs[:2], 0, 1e-10, 0, pkg.MCD_F64)
    ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_POOL)
    # the pool form solves instances of any size; a context without a basis
    # and bad arguments still fail, naming the instance
    with pytest.raises(pkg.MCDError) as e:
        pkg.mcd_batch_lanczos_ground([ctxs[0], nob], 50, 1e-10, 0, pkg.MCD_F64)
    assert e.value.status == -8 and "instance 1" in str(e.value)
    with pytest.raises(pkg.MCDError) as e:
        pkg.mcd_batch_lanczos_ground(ctxs[:2], 0, 1e-10, 0, pkg.MCD_F64)
    assert e.value.status == -1


@pytest.mark.slow
def test_batch_256_impurities():
    # the batched workload: 256 instances, bases log-uniform in [1e3, 1e5]
    ms = IM.batch(256)
    ctxs = [make_ctx(m) for m in ms]
    r = pkg.mcd_batch_lanczos_ground(ctxs, 400, 1e-10, 0, pkg.MCD_F32, allow_not_converged=True)
    rng = np.random.default_rng(0)
    for i in rng.choice(256, 8, replace=False):
        s = ctxs[i].mcd_lanczos_ground(400, 1e-10, 0, pkg.MCD_F64, allow_not_converged=True)
        assert abs(r["E0"][i] - s["E0"]) < 1e-6
