"""Green functions and their gradients for a batch of impurity models (the
batched workload: 2x2 plaquette + 8 bath sites, uneven Monte Carlo bases)
through the C ABI: G(i omega_n) on 64 Matsubara points at beta_M = 50 for the
cluster's spin-up orbitals, every instance run concurrently
(mcd_batch_band_lanczos_green) from the ground states mcd_batch_lanczos_ground
leaves in each context:
- equal bit for bit to the one-instance call on the same context;
- against the oracle's block-Krylov G from the oracle's own ground state on
  the smaller instances;
- the batched gradient (mcd_batch_green_gradient) equal bit for bit to the
  one-instance gradient, with the bath parameters' parts read out of it;
- argument errors (a context twice) and a failing instance reported by index."""
import numpy as np
import pytest

import paper_2509_22975_gb300 as pkg
from oracle import green as G, hamiltonian as H, lanczos as LZ
from workloads import impurity as IM

pytestmark = pytest.mark.gpu
ORB = [(0, 0), (1, 0), (2, 0), (3, 0)]
Z = 1j * (2 * np.arange(64) + 1) * np.pi / 50.0


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def make_ctx(m):
    ctx = pkg.Context(0)
    ctx.mcd_set_hamiltonian(m.t, m.eps, m.U_sites, m.n_up, m.n_dn)
    ctx.mcd_build_basis(m.seed, m.n_f, m.beta, [m.seed_word()])
    return ctx


@pytest.fixture(scope="module")
def batch():
    ms = IM.batch(12)
    ms[0].n_f, ms[1].n_f, ms[2].n_f = 1200, 900, 2500   # small ones the oracle handles
    ctxs = [make_ctx(m) for m in ms]
    r = pkg.mcd_batch_lanczos_ground(ctxs, 800, 1e-13, 0, pkg.MCD_F64)
    return ms, ctxs, r


@pytest.mark.parametrize("dtype", [pkg.MCD_F64, pkg.MCD_F32])
def test_batched_green_equals_single_instance_calls(batch, dtype):
    ms, ctxs, _ = batch
    Gb, dp, dm = pkg.mcd_batch_band_lanczos_green(ctxs, ORB, 40, 1.0, Z, dtype=dtype)
    assert Gb.shape == (len(ctxs), len(Z), 4, 4)
    for i, c in enumerate(ctxs):
        Gi, dpi, dmi = c.mcd_band_lanczos_green(ORB, 40, 1.0, Z, dtype=dtype)
        assert (dpi, dmi) == (dp[i], dm[i])
        assert np.array_equal(Gi, Gb[i])


def test_batched_green_against_the_oracle(batch):
    ms, ctxs, r = batch
    Gb, dp, dm = pkg.mcd_batch_band_lanczos_green(ctxs[:3], ORB, 40, 1.0, Z)
    for i in range(3):
        m = ms[i]
        B = ctxs[i].mcd_get_basis()
        M = H.Model(m.n_sites, m.t, m.eps, m.U_sites)
        E_ref, v_ref, _ = LZ.dense_ground(H.build(M, B).dense())
        assert abs(r["E0"][i] - E_ref) < 1e-10 * abs(E_ref)
        ref = G.green(M, B, v_ref, E_ref, ORB, 40, 1.0, Z)
        assert (dp[i], dm[i]) == (ref.plus.dim, ref.minus.dim)
        err = np.max(np.abs(Gb[i] - ref.G)) / np.max(np.abs(ref.G))
        assert err < 1e-8, (i, err)


def test_batched_gradient_equals_single_instance_gradients(batch):
    ms, ctxs, _ = batch
    sub = ctxs[:4]
    rng = np.random.default_rng(11)
    gG = rng.normal(size=(len(sub), 8, 4, 4)) + 1j * rng.normal(size=(len(sub), 8, 4, 4))
    z = Z[:8]
    gt, ge, gu, its = pkg.mcd_batch_green_gradient(sub, ORB, 30, 1.0, z, gG)
    for i, c in enumerate(sub):
        t1, e1, u1, it1 = c.mcd_green_gradient(ORB, 30, 1.0, z, gG[i])
        assert np.array_equal(t1, gt[i]) and np.array_equal(e1, ge[i]) and np.array_equal(u1, gu[i])
        assert it1 == its[i]
        # the bath parameters: bath energies (sites 4..11) and hybridisations
        # (cluster-bath bonds), all nonzero in general
        hyb = gt[i][:4, 4:]
        assert np.all(np.isfinite(ge[i][4:])) and np.count_nonzero(hyb) == 32


def test_batched_errors(batch):
    ms, ctxs, _ = batch
    with pytest.raises(pkg.MCDError) as e:
        pkg.mcd_batch_band_lanczos_green([ctxs[0], ctxs[0]], ORB, 10, 1.0, Z[:2])
    assert e.value.status == -1
    fresh = make_ctx(ms[5])                     # no ground state yet: instance 1 fails
    with pytest.raises(pkg.MCDError) as e:
        pkg.mcd_batch_band_lanczos_green([ctxs[0], fresh], ORB, 10, 1.0, Z[:2])
    assert e.value.status == -8 and "instance 1" in str(e.value)
