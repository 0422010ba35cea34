"""Pins of the oracle's Hamiltonian, signs and Lanczos against facts fixed
outside the oracle: closed forms, the paper's printed full-ED energies,
particle-hole symmetry, brute-force Jordan-Wigner operator products and a
library eigensolver."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fock, hamiltonian as H, lanczos as LZ
from workloads import lattice as L

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def model(lat, U, mu=0.0, eps=None):
    n = lat.n_sites
    e = np.full(n, -mu) if eps is None else np.asarray(eps, float)
    Uv = np.full(n, float(U)) if np.isscalar(U) else np.asarray(U, float)
    return H.Model(n, lat.t, e, Uv)


def ground(lat, U, n_up, n_dn, mu=0.0):
    P = H.build(model(lat, U, mu), fock.sector(lat.n_sites, n_up, n_dn))
    if P.n <= 2000:
        return LZ.dense_ground(P.dense())[0]
    A = P.sparse()
    return LZ.lanczos(lambda v: A @ v, P.n, max_iter=600, tol=1e-13).E0


def trunc4(x):
    """The paper prints its energies truncated (not rounded) to 4 decimals."""
    return math.trunc(x * 1e4) / 1e4


# --- closed forms -------------------------------------------------------------
@pytest.mark.parametrize("U", [0.0, 1.0, 4.0, 8.0, 12.5])
def test_dimer_closed_form(U):
    # Two sites, one bond t_01 = -t, one electron of each spin:
    # E0 = (U - sqrt(U^2 + 16 t^2)) / 2.
    E = ground(L.dimer(1.0), U, 1, 1)
    assert abs(E - (U - math.sqrt(U * U + 16.0)) / 2) < 1e-12


@pytest.mark.parametrize("nc,n_up,n_dn", [(8, 4, 4), (8, 3, 5), (6, 2, 3), (10, 5, 5)])
def test_free_fermions(nc, n_up, n_dn):
    # U = 0 on a ring: the single-particle energies are -2 t cos(2 pi k / N);
    # the many-body ground state fills the lowest ones for each spin.
    e = sorted(-2.0 * math.cos(2 * math.pi * k / nc) for k in range(nc))
    exact = sum(e[:n_up]) + sum(e[:n_dn])
    assert abs(ground(L.ring(nc), 0.0, n_up, n_dn) - exact) < 1e-10


# --- the paper's printed full-ED energies ---------------------------------------
@pytest.mark.parametrize("nc", [4, 8])
def test_paper_ring_energies(nc):
    ref = json.load(open(os.path.join(GOLD, "paper_energies.json")))["ring"][str(nc)]
    E = ground(L.ring(nc), 8.0, nc // 2, nc // 2, mu=4.0)
    assert trunc4(E / nc) == ref


@pytest.mark.slow
def test_paper_ring12_energy():
    ref = json.load(open(os.path.join(GOLD, "paper_energies.json")))["ring"]["12"]
    E = ground(L.ring(12), 8.0, 6, 6, mu=4.0)
    assert trunc4(E / 12) == ref


def test_paper_square8_energy():
    g = json.load(open(os.path.join(GOLD, "paper_energies.json")))["square"]["4x2"]
    lat = L.superlattice_cluster(tuple(g["R1"]), tuple(g["R2"]))
    E = ground(lat, 8.0, g["n_up"], g["n_dn"], mu=4.0)
    assert trunc4(E / 8) == g["value"]


@pytest.mark.slow
def test_paper_square12_energy():
    g = json.load(open(os.path.join(GOLD, "paper_energies.json")))["square"]["12"]
    lat = L.superlattice_cluster(tuple(g["R1"]), tuple(g["R2"]))
    E = ground(lat, 8.0, g["n_up"], g["n_dn"], mu=4.0)
    assert trunc4(E / 12) == g["value"]


def test_paper_square4_row_is_the_ring():
    ref = json.load(open(os.path.join(GOLD, "paper_energies.json")))["ring"]["4"]
    assert trunc4(ground(L.ring(4), 8.0, 2, 2, mu=4.0) / 4) == ref


def test_afm_labels():
    g = json.load(open(os.path.join(GOLD, "paper_energies.json")))["afm_labels"]
    lat = L.ring(4)
    w = L.afm_seed(lat, 2, 2)
    assert w == 90
    assert (int(g["90"]["up"], 2) << 4) | int(g["90"]["dn"], 2) == 90
    assert (int(g["165"]["up"], 2) << 4) | int(g["165"]["dn"], 2) == 165


def test_four_site_sector_structure():
    # App. D: the 4-site, N_e = 4, S_z = 0 sector is 36 x 36; nonzero
    # off-diagonal entries are hoppings of magnitude t, the diagonal holds
    # multiples of U (mu = 0 there).
    dim = json.load(open(os.path.join(GOLD, "paper_energies.json")))["four_site_sector"]["dim"]
    P = H.build(model(L.ring(4), 8.0), fock.sector(4, 2, 2))
    D = P.dense()
    assert D.shape == (dim, dim)
    off = D[~np.eye(dim, dtype=bool)]
    assert set(np.unique(np.abs(off[off != 0]))) == {1.0}
    assert set(np.unique(np.diag(D))) <= {0.0, 8.0, 16.0}


# --- particle-hole symmetry -------------------------------------------------------
@pytest.mark.parametrize("n_up,n_dn", [(3, 3), (2, 3), (1, 4)])
def test_particle_hole(n_up, n_dn):
    # c_{i s} -> (-1)^i c^dag_{i s} maps the bipartite ring's (N_up, N_dn)
    # sector onto (N - N_up, N - N_dn) with E shifted by U (N - N_up - N_dn).
    nc, U = 8, 4.0
    lat = L.ring(nc)
    E1 = ground(lat, U, n_up, n_dn)
    E2 = ground(lat, U, nc - n_up, nc - n_dn)
    assert abs(E2 - (E1 + U * (nc - n_up - n_dn))) < 1e-10


# --- brute-force Jordan-Wigner operators -------------------------------------------
def jw_annihilators(n):
    """c_m on the full 4^n Fock space, indexed by word (up << n) | dn; mode
    order up 0..n-1 then down 0..n-1; sign = (-1)^(occupied modes before m),
    counted mode by mode."""
    dim = 1 << (2 * n)
    pos = [n + m for m in range(n)] + [m for m in range(n)]   # bit of mode m
    ops = []
    for m in range(2 * n):
        rows, cols, vals = [], [], []
        for w in range(dim):
            if not (w >> pos[m]) & 1:
                continue
            before = sum((w >> pos[k]) & 1 for k in range(m))
            rows.append(w ^ (1 << pos[m]))
            cols.append(w)
            vals.append((-1.0) ** before)
        ops.append(sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim)))
    return ops


def brute_hamiltonian(n, t, eps, U):
    c = jw_annihilators(n)
    cu, cd = c[:n], c[n:]
    Hf = sp.csr_matrix((1 << (2 * n), 1 << (2 * n)))
    for s in (cu, cd):
        for i in range(n):
            for j in range(n):
                if i != j and t[i, j] != 0:
                    Hf = Hf + t[i, j] * (s[i].T @ s[j])
            Hf = Hf + eps[i] * (s[i].T @ s[i])
    for i in range(n):
        Hf = Hf + U[i] * ((cu[i].T @ cu[i]) @ (cd[i].T @ cd[i]))
    return Hf.tocsr()


@pytest.mark.parametrize("n,n_up,n_dn", [(4, 2, 2), (5, 2, 3), (5, 3, 1), (6, 3, 3)])
def test_signs_against_operator_products(n, n_up, n_dn):
    rng = np.random.default_rng(100 + n)
    t = rng.normal(size=(n, n))
    t = t + t.T
    np.fill_diagonal(t, 0.0)
    t[rng.random((n, n)) < 0.2] = 0.0
    t = np.triu(t, 1)
    t = t + t.T
    eps, U = rng.normal(size=n), rng.uniform(0, 8, size=n)
    Hf = brute_hamiltonian(n, t, eps, U)
    basis = fock.sector(n, n_up, n_dn)
    idx = basis.astype(np.int64)
    ref = Hf[idx][:, idx].toarray()
    got = H.build(H.Model(n, t, eps, U), basis).dense()
    assert np.array_equal(got, ref) or np.max(np.abs(got - ref)) < 1e-14
    # a truncated basis gives exactly the principal submatrix (App. B:
    # discarding out-of-basis states == projecting H)
    sub = np.sort(rng.choice(len(basis), size=max(2, len(basis) // 3), replace=False))
    gs = H.build(H.Model(n, t, eps, U), basis[sub]).dense()
    assert np.max(np.abs(gs - ref[np.ix_(sub, sub)])) < 1e-14


# --- projection and Lanczos ----------------------------------------------------------
def test_projected_is_symmetric_and_exact_apply():
    lat = L.ring(8)
    rng = np.random.default_rng(3)
    full = fock.sector(8, 4, 4)
    sub = np.sort(rng.choice(len(full), 700, replace=False))
    P = H.build(model(lat, 4.0, 0.3), full[sub])
    D = P.dense()
    assert np.array_equal(D, D.T)
    x = rng.normal(size=(P.n, 3))
    y = H.apply_exact(P, x)
    assert np.max(np.abs(y - D @ x)) <= 1e-13 * np.max(np.abs(D) @ np.abs(x))


def test_lanczos_matches_dense_and_variational_bound():
    lat = L.ring(8)
    full = fock.sector(8, 4, 4)
    E_full = ground(lat, 4.0, 4, 4)
    rng = np.random.default_rng(5)
    prev = None
    for m in (500, 1500, 3000):
        sub = np.sort(rng.choice(len(full), m, replace=False)) if prev is None else \
            np.sort(np.concatenate([prev, rng.choice(np.setdiff1d(np.arange(len(full)), prev),
                                                      m - len(prev), replace=False)]))
        P = H.build(model(lat, 4.0), full[sub])
        A = P.sparse()
        Ed, vd, _ = LZ.dense_ground(P.dense())
        r = LZ.lanczos(lambda v: A @ v, P.n, max_iter=P.n, tol=1e-13, want_vector=True)
        assert abs(r.E0 - Ed) < 1e-10 * abs(Ed)
        assert r.residual < 1e-8
        assert abs(abs(r.psi @ vd) - 1.0) < 1e-8
        assert r.E0 >= E_full - 1e-12                     # Omega~ >= Omega
        if prev is not None:
            assert r.E0 <= E_prev + 1e-12                 # nested bases: non-increasing
        prev, E_prev = sub, r.E0


def test_lanczos_tridiagonal_is_orthogonal_projection():
    # The recursion's coefficients are those of an orthonormal Krylov basis:
    # for a few steps (no loss of orthogonality yet) V^T H V equals the
    # tridiagonal matrix built from a_n, b_n.
    lat = L.ring(6)
    P = H.build(model(lat, 3.0), fock.sector(6, 3, 3))
    D = P.dense()
    r = LZ.lanczos(lambda v: D @ v, P.n, max_iter=8, tol=0.0, want_vector=False)
    V = []
    phi = LZ.start_vector(P.n, 0)
    prev = np.zeros(P.n)
    nn_prev = 1.0
    for it in range(8):
        nn = phi @ phi
        V.append(phi / np.sqrt(nn))
        Hp = D @ phi
        a = phi @ Hp / nn
        b2 = nn / nn_prev if it else 0.0
        phi, prev, nn_prev = Hp - a * phi - b2 * prev, phi, nn
    V = np.array(V).T
    T = np.diag(r.a) + np.diag(r.b[1:], 1) + np.diag(r.b[1:], -1)
    assert np.max(np.abs(V.T @ D @ V - T)) < 1e-9


def test_hellmann_feynman_U():
    # dE0/dU = <Omega| sum_i n_i,up n_i,dn |Omega> (pins the U term's coefficient).
    lat = L.ring(6)
    basis = fock.sector(6, 3, 3)
    U, h = 3.0, 1e-5
    Ep = LZ.dense_ground(H.build(model(lat, U + h), basis).dense())[0]
    Em = LZ.dense_ground(H.build(model(lat, U - h), basis).dense())[0]
    _, v, _ = LZ.dense_ground(H.build(model(lat, U), basis).dense())
    nU = fock.double_occupancy(basis, 6).astype(float)
    assert abs((Ep - Em) / (2 * h) - float(v @ (nU * v))) < 1e-7
