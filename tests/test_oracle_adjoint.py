"""Pins of the oracle's parameter derivatives: Euler's identity for a
Hamiltonian linear in its parameters, and Hellmann-Feynman against finite
differences of the dense ground-state energy for t, eps and U."""
import numpy as np

from oracle import fock, hamiltonian as H, lanczos as LZ
from workloads import lattice as L


def test_euler_identity():
    # sum_theta theta * d<u,Hv>/dtheta = <u, H v> (H is homogeneous of degree 1)
    lat = L.superlattice_cluster((4, 0), (0, 2), tp=-0.3)
    n = 8
    rng = np.random.default_rng(0)
    M = H.Model(n, lat.t, rng.normal(size=n), rng.uniform(2, 6, n))
    B = fock.sector(n, 4, 3)[::5]
    u, v = rng.normal(size=(len(B), 2)), rng.normal(size=(len(B), 2))
    gt, ge, gu = H.parameter_derivatives(M, B, u, v)
    lhs = 0.5 * np.sum(lat.t * gt) + M.eps @ ge + M.U @ gu
    rhs = np.sum(u * (H.build(M, B).sparse() @ v))
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_hellmann_feynman_all_parameters():
    lat = L.ring(6)
    n = 6
    rng = np.random.default_rng(1)
    eps, U = rng.normal(size=n) * 0.3, rng.uniform(2, 5, n)
    B = fock.sector(n, 3, 2)

    def E(t, e, u):
        return LZ.dense_ground(H.build(H.Model(n, t, e, u), B).dense())[0]

    _, psi, _ = LZ.dense_ground(H.build(H.Model(n, lat.t, eps, U), B).dense())
    gt, ge, gu = H.parameter_derivatives(H.Model(n, lat.t, eps, U), B, psi, psi)
    h = 1e-5
    T = lat.t.copy()
    T[0, 1] += h
    T[1, 0] += h
    Tm = lat.t.copy()
    Tm[0, 1] -= h
    Tm[1, 0] -= h
    assert abs((E(T, eps, U) - E(Tm, eps, U)) / (2 * h) - gt[0, 1]) < 1e-7
    for i in (0, 3):
        d = np.zeros(n)
        d[i] = h
        assert abs((E(lat.t, eps + d, U) - E(lat.t, eps - d, U)) / (2 * h) - ge[i]) < 1e-7
        assert abs((E(lat.t, eps, U + d) - E(lat.t, eps, U - d)) / (2 * h) - gu[i]) < 1e-7
