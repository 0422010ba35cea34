"""Gradient of the Green function with respect to (t_ij, eps_i, U_i) through
the C ABI (mcd_green_gradient): against the oracle's dense gradient (spin-up
and spin-down orbitals, site-dependent U, a truncated ground state), against
central finite differences of the device G on an impurity model, and through
torch.autograd."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from paper_2509_22975_gb300 import autograd as AG
from oracle import fock, green as G, hamiltonian as H
from workloads import impurity as IM, lattice as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def ground(ctx):
    """fp64 Lanczos ground state, kept by the context (a psi buffer is passed)."""
    n = ctx.mcd_basis_info(nnz=False)["n_states"]
    psi = torch.empty(n, dtype=torch.float64, device="cuda:0")
    return ctx.mcd_lanczos_ground(1000, 1e-13, 0, pkg.MCD_F64, psi=psi)


def ctx_for(M, n_up, n_dn, basis):
    ctx = pkg.Context(0)
    ctx.mcd_set_hamiltonian(M.t, M.eps, M.U, n_up, n_dn)
    ctx.mcd_set_basis(basis)
    ground(ctx)
    return ctx


def compare(ctx, M, B, orb, w_t, z, rng, nb=200, tol=1e-7):
    gR = rng.normal(size=(len(z), len(orb), len(orb)))
    gI = rng.normal(size=(len(z), len(orb), len(orb)))
    gt, ge, gu, it = ctx.mcd_green_gradient(orb, nb, w_t, z, gR + 1j * gI)
    rt, re, ru = G.green_gradient(M, B, orb, w_t, z, gR, gI)
    scale = max(np.max(np.abs(rt)), np.max(np.abs(re)), np.max(np.abs(ru)), 1.0)
    for a, b in ((gt, rt), (ge, re), (gu, ru)):
        assert np.max(np.abs(a - b)) < tol * scale, np.max(np.abs(a - b)) / scale
    assert np.all(gt[M.t == 0] == 0)
    return it


def test_ring_spin_up_against_oracle():
    n = 6
    M = H.Model(n, L.ring(n).t, np.full(n, -2.0), np.full(n, 4.0))
    B = fock.sector(n, 3, 3)
    ctx = ctx_for(M, 3, 3, B)
    compare(ctx, M, B, [(0, 0), (2, 0)], 1.0, np.array([0.7j, 0.2 + 1.1j]), np.random.default_rng(2))


def test_random_model_spin_down_site_dependent_u():
    n = 6
    rng = np.random.default_rng(3)
    t = np.zeros((n, n))
    for i, j in [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (0, 3), (1, 4)]:
        t[i, j] = t[j, i] = rng.normal()
    M = H.Model(n, t, rng.uniform(-1, 1, n), rng.uniform(0, 5, n))
    B = fock.sector(n, 3, 2)
    ctx = ctx_for(M, 3, 2, B)
    compare(ctx, M, B, [(1, 1), (4, 1), (5, 1)], 1.0, np.array([0.9j, 2.1j, 0.5 + 0.3j]), rng)


def test_truncated_ground_state():
    n = 6
    rng = np.random.default_rng(5)
    t = np.zeros((n, n))
    for i, j in [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (0, 3)]:
        t[i, j] = t[j, i] = -1.0 + 0.3 * rng.normal()
    M = H.Model(n, t, rng.uniform(-1, 1, n), np.full(n, 3.0))
    B = fock.sector(n, 3, 3)
    w, V = np.linalg.eigh(H.build(M, B).dense())
    p = np.sort(V[:, 0] ** 2)[::-1]
    cum = np.cumsum(p)
    k = next(k for k in range(len(p) // 2, len(p) - 1) if p[k] > 1.01 * p[k + 1])
    w_t = (cum[k - 1] + 0.5 * p[k]) / cum[-1]
    ctx = ctx_for(M, 3, 3, B)
    compare(ctx, M, B, [(0, 0), (1, 0)], w_t, np.array([0.8j]), rng)


def test_impurity_finite_differences_of_device_green():
    # bath energies, hybridisations and the cluster U of an impurity model on
    # a Monte Carlo basis; S(theta +- h) from the device G itself
    m = IM.impurity(3, n_f=400)
    ctx = pkg.Context(0)
    ctx.mcd_set_hamiltonian(m.t, m.eps, m.U_sites, m.n_up, m.n_dn)
    ctx.mcd_build_basis(m.seed, m.n_f, m.beta, [m.seed_word()])
    B = ctx.mcd_get_basis()
    orb = [(0, 0), (1, 0), (2, 0), (3, 0)]
    beta_m = 50.0
    z = 1j * (2 * np.arange(6) + 1) * np.pi / beta_m
    nb = 150
    rng = np.random.default_rng(7)
    g = rng.normal(size=(len(z), 4, 4)) + 1j * rng.normal(size=(len(z), 4, 4))

    def S(t, eps, U):
        c = pkg.Context(0)
        c.mcd_set_hamiltonian(t, eps, U, m.n_up, m.n_dn)
        c.mcd_set_basis(B)
        ground(c)
        Gz, _, _ = c.mcd_band_lanczos_green(orb, nb, 1.0, z)
        return float(np.sum(g.real * Gz.real + g.imag * Gz.imag))

    ground(ctx)
    gt, ge, gu, _ = ctx.mcd_green_gradient(orb, nb, 1.0, z, g)
    h = 1e-5
    for b in (4, 9):                                    # bath energies
        d = np.zeros(12)
        d[b] = h
        fd = (S(m.t, m.eps + d, m.U_sites) - S(m.t, m.eps - d, m.U_sites)) / (2 * h)
        assert abs(fd - ge[b]) < 1e-6 * max(1.0, abs(ge[b])), (b, fd, ge[b])
    for i, b in ((0, 4), (2, 7), (3, 11)):              # hybridisations
        d = np.zeros((12, 12))
        d[i, b] = d[b, i] = h
        fd = (S(m.t + d, m.eps, m.U_sites) - S(m.t - d, m.eps, m.U_sites)) / (2 * h)
        assert abs(fd - gt[i, b]) < 1e-6 * max(1.0, abs(gt[i, b])), (i, b, fd, gt[i, b])
    d = np.zeros(12)
    d[:4] = h                                           # the cluster U (one value on four sites)
    fd = (S(m.t, m.eps, m.U_sites + d) - S(m.t, m.eps, m.U_sites - d)) / (2 * h)
    assert abs(fd - gu[:4].sum()) < 1e-6 * max(1.0, abs(gu[:4].sum()))


def test_autograd_matches_direct_call():
    n = 6
    M = H.Model(n, L.ring(n).t, np.full(n, -2.0), np.full(n, 4.0))
    B = fock.sector(n, 3, 3)
    ctx = pkg.Context(0)
    ctx.mcd_set_hamiltonian(M.t, M.eps, M.U, 3, 3)
    ctx.mcd_set_basis(B)
    orb = [(0, 0), (3, 0)]
    z = np.array([0.6j, 1.4j])
    t = torch.tensor(M.t, dtype=torch.float64, requires_grad=True)
    eps = torch.tensor(M.eps, dtype=torch.float64, requires_grad=True)
    U = torch.tensor(4.0, dtype=torch.float64, requires_grad=True)
    Gt = AG.green(ctx, t, eps, U, orb, 200, 1.0, z)
    w = torch.from_numpy(np.random.default_rng(9).normal(size=tuple(Gt.shape)))
    (Gt * w).sum().backward()
    gt, ge, gu, _ = ctx.mcd_green_gradient(orb, 200, 1.0, z, w[..., 0].numpy() + 1j * w[..., 1].numpy())
    assert np.allclose(t.grad.numpy(), gt, atol=1e-12)
    assert np.allclose(eps.grad.numpy(), ge, atol=1e-12)
    assert abs(U.grad.item() - gu.sum()) < 1e-12 * max(1.0, abs(gu.sum()))


def test_errors():
    n = 6
    M = H.Model(n, L.ring(n).t, np.full(n, -2.0), np.full(n, 4.0))
    ctx = pkg.Context(0)
    ctx.mcd_set_hamiltonian(M.t, M.eps, M.U, 3, 3)
    ctx.mcd_set_basis(fock.sector(n, 3, 3))
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_green_gradient([(0, 0)], 10, 1.0, [1j], np.ones((1, 1, 1)))
    assert e.value.status == -8                          # no ground state
    ground(ctx)
    with pytest.raises(pkg.MCDError):
        ctx.mcd_green_gradient([(0, 0), (1, 1)], 10, 1.0, [1j], np.ones((1, 2, 2)))   # mixed spins
    with pytest.raises(pkg.MCDError):
        ctx.mcd_green_gradient([(0, 0)], 10, 1.0, [1j], np.ones((1, 1, 1)), cg_tol=0.0)
