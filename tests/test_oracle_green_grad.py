"""Pins of the oracle's gradient of the Green function with respect to the
Hamiltonian's parameters (oracle.green.green_gradient), against things other
than itself: the free-fermion closed form dG = R (dh) R with R = (z - h)^-1
of the single-particle matrix h, and central finite differences of the
oracle's exact G (interacting, with and without target-weight truncation)."""
import numpy as np
import pytest

from oracle import fock, green as G, hamiltonian as H
from workloads import lattice as L


def S_of(model, basis, orb, w_t, z, gR, gI):
    """The scalar whose gradient is taken: sum gR Re G + gI Im G (exact G)."""
    Hd = H.build(model, basis).dense()
    w, V = np.linalg.eigh(Hd)
    res = G.green(model, basis, V[:, 0], float(w[0]), orb, 0, 1.0 if w_t is None else w_t, z, exact=True)
    return float(np.sum(gR * res.G.real + gI * res.G.imag)), res.keep


def random_g(rng, nz, L_):
    return rng.normal(size=(nz, L_, L_)), rng.normal(size=(nz, L_, L_))


def test_free_fermions_closed_form():
    # U = 0, full sector: G(z) = (z - h)^-1 on the single-particle orbitals,
    # so dS/dh_ij = Re sum conj(g) . R (e_i e_j^T + e_j e_i^T) R
    n = 6
    lat = L.ring(n)
    eps = np.array([0.1, -0.2, 0.05, 0.3, -0.1, 0.0])
    M = H.Model(n, lat.t, eps, np.zeros(n))
    B = fock.sector(n, 3, 3)
    orb = [(i, 0) for i in range(n)]
    z = np.array([0.5j, 1.3j, 0.4 + 0.9j])
    rng = np.random.default_rng(1)
    gR, gI = random_g(rng, len(z), n)
    gt, ge, gu = G.green_gradient(M, B, orb, 1.0, z, gR, gI)
    h = lat.t + np.diag(eps)
    gc = gR + 1j * gI
    for i in range(n):
        ref = 0.0
        for iz, zz in enumerate(z):
            R = np.linalg.inv(zz * np.eye(n) - h)
            ref += np.sum(np.real(np.conj(gc[iz]) * np.outer(R[:, i], R[i, :])))
        assert abs(ge[i] - ref) < 1e-9 * max(1.0, abs(ref))
    for i in range(n):
        for j in range(i + 1, n):
            if lat.t[i, j] == 0:
                assert gt[i, j] == 0.0
                continue
            ref = 0.0
            for iz, zz in enumerate(z):
                R = np.linalg.inv(zz * np.eye(n) - h)
                ref += np.sum(np.real(np.conj(gc[iz]) * (np.outer(R[:, i], R[j, :]) + np.outer(R[:, j], R[i, :]))))
            assert abs(gt[i, j] - ref) < 1e-9 * max(1.0, abs(ref))


def finite_difference_check(M, B, orb, w_t, z, rng, h=1e-5, tol=2e-6):
    gR, gI = random_g(rng, len(z), len(orb))
    gt, ge, gu = G.green_gradient(M, B, orb, w_t, z, gR, gI)
    _, keep0 = S_of(M, B, orb, w_t, z, gR, gI)
    for par in G.parameters(M):
        um = G.unit_model(M.n, par)
        Mp = H.Model(M.n, M.t + h * um.t, M.eps + h * um.eps, M.U + h * um.U)
        Mm = H.Model(M.n, M.t - h * um.t, M.eps - h * um.eps, M.U - h * um.U)
        Sp, kp = S_of(Mp, B, orb, w_t, z, gR, gI)
        Sm, km = S_of(Mm, B, orb, w_t, z, gR, gI)
        assert np.array_equal(kp, keep0) and np.array_equal(km, keep0)   # kept set fixed
        fd = (Sp - Sm) / (2 * h)
        kind, i, j = par
        an = gt[i, j] if kind == "t" else (ge[i] if kind == "eps" else gu[i])
        assert abs(fd - an) < tol * max(1.0, abs(an)), (par, fd, an)


def test_interacting_ring_finite_differences():
    n = 6
    lat = L.ring(n)
    M = H.Model(n, lat.t, np.full(n, -2.0), np.full(n, 4.0))
    B = fock.sector(n, 3, 3)
    finite_difference_check(M, B, [(0, 0), (2, 0)], 1.0, np.array([0.7j, 0.2 + 1.1j]), np.random.default_rng(2))


def test_random_model_site_dependent_u_finite_differences():
    n = 6
    rng = np.random.default_rng(3)
    t = np.zeros((n, n))
    for i, j in [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (0, 3), (1, 4)]:
        t[i, j] = t[j, i] = rng.normal()
    M = H.Model(n, t, rng.uniform(-1, 1, n), rng.uniform(0, 5, n))
    B = fock.sector(n, 3, 2)
    finite_difference_check(M, B, [(1, 1), (4, 1), (5, 1)], 1.0, np.array([0.9j, 2.1j]), rng)


def test_truncated_ground_state_finite_differences():
    # w_t < 1: the renormalised truncated ground state is differentiated
    # through P Omega / |P Omega|; an asymmetric model and a w_t inside a gap
    # between distinct weights keep the kept words the same under +-h
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
    finite_difference_check(M, B, [(0, 0), (1, 0)], w_t, np.array([0.8j]), rng)
