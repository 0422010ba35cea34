"""Pins of the oracle's Green function (Sec. "Subspace of the Green
function", App. C): the non-interacting closed form, the anticommutator sum
rule, the 1/z tail, particle-hole symmetry of the DOS, Krylov exhaustion
against the dense Lehmann sum, and the target-weight truncation rule."""
import numpy as np
import pytest

from oracle import fock, green as G, hamiltonian as H, lanczos as LZ
from workloads import lattice as L


def ground(M, basis):
    E0, psi, _ = LZ.dense_ground(H.build(M, basis).dense())
    return E0, psi


def test_free_fermion_closed_form():
    # U = 0, 6-ring, 3 + 3 electrons (closed shell): G_ij(z) = [(z - (T - mu))^-1]_ij
    n, mu = 6, 0.3
    lat = L.ring(n)
    M = H.Model(n, lat.t, np.full(n, -mu), np.zeros(n))
    B = fock.sector(n, 3, 3)
    E0, psi = ground(M, B)
    orb = [(i, 0) for i in range(n)]
    z = np.array([0.1 + 0.05j, 1.3 + 0.2j, -2.0 + 0.5j, 3.0j])
    r = G.green(M, B, psi, E0, orb, 50, 1.0, z)
    h1 = lat.t - mu * np.eye(n)
    ref = np.array([np.linalg.inv(zz * np.eye(n) - h1) for zz in z])
    assert np.max(np.abs(r.G - ref)) < 1e-10


@pytest.mark.parametrize("w_t", [1.0, 0.9])
def test_sum_rule_and_tail_on_a_truncated_mc_basis(w_t):
    # sum_m Q+ Q+^T + sum_n Q- Q-^T = <{c_mu, c^dag_nu}> = delta_mu nu, exactly,
    # for any basis: c^dag |Omega~> lies in span F~+ by construction.
    from oracle import sampler as S
    n, U = 8, 4.0
    lat = L.ring(n)
    M = H.Model(n, lat.t, np.full(n, -U / 2), np.full(n, U))
    seed = L.afm_seed(lat, 4, 4)
    B = S.sample_basis(n, lat.t, np.full(n, U), 4, 4, 1200, 0.4, [seed], seed=3)
    E0, psi = ground(M, B)
    orb = [(i, 0) for i in range(n)]
    r = G.green(M, B, psi, E0, orb, 12, w_t, np.array([1e7j]))
    Sr = r.plus.Q @ r.plus.Q.T + r.minus.Q @ r.minus.Q.T
    assert np.max(np.abs(Sr - np.eye(n))) < 1e-12
    # z G(z) -> identity as |z| -> infinity
    assert np.max(np.abs(1e7j * r.G[0] - np.eye(n))) < 1e-5


def test_exhausted_krylov_equals_dense_lehmann():
    n, U = 6, 3.0
    lat = L.ring(n)
    M = H.Model(n, lat.t, np.full(n, -1.0), np.full(n, U))
    B = fock.sector(n, 3, 2)
    E0, psi = ground(M, B)
    orb = [(0, 1), (2, 1), (3, 1)]
    z = np.linspace(-5, 5, 9) + 0.1j
    rk = G.green(M, B, psi, E0, orb, 200, 1.0, z)
    rx = G.green(M, B, psi, E0, orb, 0, 1.0, z, exact=True)
    assert np.max(np.abs(rk.G - rx.G)) < 1e-11


def test_particle_hole_symmetric_dos_at_half_filling():
    # bipartite 6-ring, mu = U/2, full sector: A(omega) = A(-omega)
    n, U = 6, 4.0
    lat = L.ring(n)
    M = H.Model(n, lat.t, np.full(n, -U / 2), np.full(n, U))
    B = fock.sector(n, 3, 3)
    E0, psi = ground(M, B)
    w = np.linspace(-6, 6, 61)
    r = G.green(M, B, psi, E0, [(i, 0) for i in range(n)], 100, 1.0, w + 0.05j)
    A = G.dos(r.G)
    assert np.max(np.abs(A - A[::-1])) < 1e-10
    assert np.all(A > 0)


def test_few_blocks_is_an_approximation_that_improves():
    n, U = 6, 4.0
    lat = L.ring(n)
    M = H.Model(n, lat.t, np.full(n, -U / 2), np.full(n, U))
    B = fock.sector(n, 3, 3)
    E0, psi = ground(M, B)
    z = np.linspace(-6, 6, 13) + 0.3j
    orb = [(i, 0) for i in range(n)]
    ex = G.green(M, B, psi, E0, orb, 0, 1.0, z, exact=True).G
    errs = [np.max(np.abs(G.green(M, B, psi, E0, orb, r, 1.0, z).G - ex)) for r in (2, 4, 8, 16)]
    assert all(a > b for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-6


def test_truncation_rule():
    rng = np.random.default_rng(1)
    psi = rng.normal(size=50)
    keep, c = G.truncate(psi, 0.9)
    p = psi / np.linalg.norm(psi)
    w = p ** 2
    # brute force: shortest set of largest weights reaching 0.9
    order = np.argsort(-w, kind="stable")
    k = next(i for i in range(1, 51) if w[order[:i]].sum() >= 0.9)
    assert np.array_equal(keep, np.sort(order[:k]))
    assert abs(np.linalg.norm(c) - 1) < 1e-14
    assert np.array_equal(G.truncate(psi, 1.0)[0], np.arange(50))
