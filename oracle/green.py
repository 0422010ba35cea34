"""Green function in the truncated excited subspaces (Sec. "Subspace of the
Green function", Sec. "Further truncation", App. C).

Steps, in the paper's order:

1. target-weight truncation: normalise |Omega~>, order its coefficients by
   |c_n|^2 (largest first; ties by basis index) and keep the shortest prefix
   whose weight reaches w_t; the kept part is renormalised (reading: the paper
   does not say whether it renormalises);
2. excited subspaces F~+ = U_mu c^dag_mu F~ and F~- = U_mu c_mu F~ (each state
   once), over the kept states;
3. start vectors |phi_nu> = c^dag_nu |Omega~> in F~+ (c_nu |Omega~> in F~-);
4. band Lanczos: an orthonormal basis of the block Krylov space
   K_r^L = span{phi, H phi, ..., H^(r-1) phi} of r blocks, and the effective
   matrix H_eff = V^T H V.  In exact arithmetic this is what band Lanczos
   builds; the oracle builds it plainly (Gram-Schmidt against every earlier
   vector, twice, dropping candidates whose norm falls below a tolerance), and
   forms H_eff explicitly instead of relying on its band structure;
5. the eigenpairs (E_m, S_m) of H_eff, Q_{mu m} = <phi_mu | V S_m> (the
   Q-matrix Eq.), and the Lehmann sums
     G+_{mu nu}(z) = sum_m Q+_{mu m} Q+_{nu m} / (z + Omega~ - E+_m),
     G-_{mu nu}(z) = sum_n Q-_{mu n} Q-_{nu n} / (z - Omega~ + E-_n),
   G = G+ + G-, A(omega) = -Im sum_mu G_mu mu(omega + i eta) / pi.

Orbitals mu = (site, spin).  All fp64.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fock
from . import hamiltonian as H


def truncate(psi: np.ndarray, w_t: float):
    """Indices of the kept coefficients (ascending) and the renormalised
    coefficients on them (Sec. "Further truncation")."""
    psi = np.asarray(psi, dtype=np.float64)
    p = psi / np.linalg.norm(psi)
    w = p * p
    order = np.lexsort((np.arange(len(w)), -w))       # weight descending, index ascending
    cum = np.cumsum(w[order])
    k = int(np.searchsorted(cum, w_t * cum[-1] * (1 - 1e-15))) + 1
    k = min(k, len(w))
    keep = np.sort(order[:k])
    c = p[keep]
    return keep, c / np.linalg.norm(c)


def excited_basis(words: np.ndarray, n: int, orbitals, dagger: bool) -> np.ndarray:
    """Sorted unique words c^dag_mu w (dagger) or c_mu w over kept words w."""
    out = set()
    for w in map(int, words):
        for site, spin in orbitals:
            r = fock.create(w, n, spin, site) if dagger else fock.annihilate(w, n, 0, spin, site)
            if r is not None:
                out.add(r[0])
    return np.array(sorted(out), dtype=np.uint64)


def start_vectors(exc: np.ndarray, words: np.ndarray, coef: np.ndarray, n: int, orbitals,
                  dagger: bool) -> np.ndarray:
    """[len(exc), L]: column nu = c^dag_nu |Omega~> (or c_nu |Omega~>) in basis exc."""
    Phi = np.zeros((len(exc), len(orbitals)))
    pos = {int(w): i for i, w in enumerate(exc)}
    for w, cw in zip(map(int, words), coef):
        for nu, (site, spin) in enumerate(orbitals):
            r = fock.create(w, n, spin, site) if dagger else fock.annihilate(w, n, 0, spin, site)
            if r is not None:
                Phi[pos[r[0]], nu] += r[1] * cw
    return Phi


def block_krylov(apply, Phi: np.ndarray, n_blocks: int, dtol: float = 1e-10):
    """Orthonormal basis V of span{Phi, H Phi, ..., H^(n_blocks-1) Phi} and
    H_eff = V^T H V.  Each candidate is orthogonalised against every earlier
    basis vector (classical Gram-Schmidt, twice) and dropped ("deflated") when
    its remaining norm is below dtol times its norm before."""
    N, L = Phi.shape
    # storage for at most L vectors per block; columns [0, k) hold the basis
    V = np.zeros((N, max(L * max(n_blocks, 1), 1)), order="F")
    k = 0

    def extend(cands):
        nonlocal k
        k0 = k
        for v in np.asarray(cands).T:
            v = np.array(v, dtype=np.float64)
            n0 = np.linalg.norm(v)
            for _ in range(2):
                B = V[:, :k]
                v = v - B @ (B.T @ v)
            nv = np.linalg.norm(v)
            if nv > dtol * max(n0, 1e-300):
                V[:, k] = v / nv
                k += 1
        return V[:, k0:k]

    blk = extend(Phi)
    for _ in range(1, n_blocks):
        if blk.shape[1] == 0:
            break
        blk = extend(np.column_stack([apply(blk[:, j]) for j in range(blk.shape[1])]))
    Vk = V[:, :k]
    HV = np.column_stack([apply(Vk[:, j]) for j in range(k)]) if k else Vk
    Heff = Vk.T @ HV
    return Vk, 0.5 * (Heff + Heff.T)


@dataclass
class Poles:
    E: np.ndarray       # eigenvalues of H_eff
    Q: np.ndarray       # [L, K]
    dim: int            # |F~+-|
    krylov_dim: int


def poles(model: H.Model, exc: np.ndarray, Phi: np.ndarray, n_blocks: int) -> Poles:
    P = H.build(model, exc)
    A = P.sparse()
    V, Heff = block_krylov(lambda v: A @ v, Phi, n_blocks)
    E, S = np.linalg.eigh(Heff)
    Q = Phi.T @ (V @ S)                 # Q_{mu m} = <phi_mu | V S_m>
    return Poles(E, Q, len(exc), V.shape[1])


def exact_poles(model: H.Model, exc: np.ndarray, Phi: np.ndarray) -> Poles:
    """All eigenpairs of H~ on the excited subspace (dense), Q = Phi^T S."""
    P = H.build(model, exc)
    E, S = np.linalg.eigh(P.dense())
    return Poles(E, Phi.T @ S, len(exc), len(exc))


def lehmann(p: Poles, E0: float, z: np.ndarray, particle: bool) -> np.ndarray:
    """[nz, L, L]: sum_m Q_mu m Q_nu m / (z + E0 - E_m) (particle) or
    / (z - E0 + E_m) (hole)."""
    z = np.asarray(z, dtype=np.complex128)
    den = (z[:, None] + E0 - p.E[None, :]) if particle else (z[:, None] - E0 + p.E[None, :])
    return np.einsum("am,bm,zm->zab", p.Q, p.Q, 1.0 / den)


@dataclass
class GreenResult:
    G: np.ndarray              # [nz, L, L] complex, G+ + G-
    plus: Poles
    minus: Poles
    keep: np.ndarray
    E0: float


def green(model: H.Model, basis: np.ndarray, psi: np.ndarray, E0: float, orbitals, n_blocks: int,
          w_t: float, z: np.ndarray, exact: bool = False) -> GreenResult:
    """G_{mu nu}(z) of Eqs. (green), (green_qmatrix) in the truncated excited
    subspaces.  Orbitals must share one spin (G is block diagonal in spin)."""
    n = model.n
    keep, coef = truncate(psi, w_t)
    words = np.asarray(basis, dtype=np.uint64)[keep]
    res = {}
    for dag in (True, False):
        exc = excited_basis(words, n, orbitals, dag)
        Phi = start_vectors(exc, words, coef, n, orbitals, dag)
        res[dag] = exact_poles(model, exc, Phi) if exact else poles(model, exc, Phi, n_blocks)
    Gp = lehmann(res[True], E0, z, True)
    Gm = lehmann(res[False], E0, z, False)
    return GreenResult(Gp + Gm, res[True], res[False], keep, E0)


def dos(G: np.ndarray) -> np.ndarray:
    """A(omega) = -(1/pi) Im sum_mu G_mu mu (Eq. DOS)."""
    return -np.imag(np.einsum("zaa->z", G)) / np.pi


def parameters(model: H.Model):
    """The Hamiltonian's parameters, in the order of the gradients: one per
    bond (i < j, t_ij != 0), then eps_i and U_i of every site.  Each entry is
    (kind, i, j) and unit(entry) is the model with that parameter alone = 1."""
    n = model.n
    out = [("t", i, j) for i in range(n) for j in range(i + 1, n) if model.t[i, j] != 0.0]
    out += [("eps", i, i) for i in range(n)] + [("U", i, i) for i in range(n)]
    return out


def unit_model(n: int, par) -> H.Model:
    kind, i, j = par
    t, e, u = np.zeros((n, n)), np.zeros(n), np.zeros(n)
    if kind == "t":
        t[i, j] = t[j, i] = 1.0
    elif kind == "eps":
        e[i] = 1.0
    else:
        u[i] = 1.0
    return H.Model(n, t, e, u)


def green_gradient(model: H.Model, basis: np.ndarray, orbitals, w_t: float, z: np.ndarray,
                   gR: np.ndarray, gI: np.ndarray):
    """Gradient of S = sum_{z, mu, nu} gR Re G_{mu nu}(z) + gI Im G_{mu nu}(z)
    with respect to (t_ij per bond, eps_i, U_i), for G computed with the exact
    resolvent in the truncated excited subspaces (the limit the band Lanczos
    reaches) and the set of kept ground-state words held fixed.

    Plain dense definition, parameter by parameter (H is linear in them):
      dE0 = <Omega| dH |Omega>                                   (Hellmann-Feynman)
      dOmega = -(H - E0)^+ (dH - dE0) |Omega>                    (first-order perturbation)
      Omega_t = P Omega / |P Omega|  =>  dOmega_t = (P dOmega - Omega_t <Omega_t|P dOmega>) / |P Omega|
      phi_nu = c^dag_nu Omega_t (particle), c_nu Omega_t (hole), linear in Omega_t
      G+ = phi^T (z + E0 - H+)^-1 phi,  G- = phi^T (z - E0 + H-)^-1 phi
      dG = dphi^T R phi + phi^T R dphi - phi^T R dA R phi,  dA = +-(dE0) -+ dH+-.
    Returns (grad_t [n, n] symmetric, 0 off the bonds, grad_eps [n], grad_U [n])."""
    n = model.n
    basis = np.asarray(basis, dtype=np.uint64)
    Hd = H.build(model, basis).dense()
    w, V = np.linalg.eigh(Hd)
    E0, Om = float(w[0]), V[:, 0]
    keep, coef = truncate(Om, w_t)
    words = basis[keep]
    Pn = float(np.linalg.norm(Om[keep]))
    pinv = (V[:, 1:] / (w[1:] - E0)) @ V[:, 1:].T
    z = np.asarray(z, dtype=np.complex128)
    gc = np.asarray(gR, dtype=np.float64) + 1j * np.asarray(gI, dtype=np.float64)   # [nz, L, L]
    sides = []
    for dag in (True, False):
        exc = excited_basis(words, n, orbitals, dag)
        Phi = start_vectors(exc, words, coef, n, orbitals, dag)
        Hs = H.build(model, exc).dense()
        sgn = 1.0 if dag else -1.0
        R = [np.linalg.inv((zz + sgn * E0) * np.eye(len(exc)) - sgn * Hs) for zz in z]
        sides.append((dag, exc, Phi, sgn, R))
    gt, ge, gu = np.zeros((n, n)), np.zeros(n), np.zeros(n)
    for par in parameters(model):
        um = unit_model(n, par)
        dH = H.build(um, basis).dense()
        dE0 = float(Om @ dH @ Om)
        dOm = -pinv @ ((dH - dE0 * np.eye(len(basis))) @ Om)
        dPt = dOm[keep]
        dcoef = (dPt - coef * float(coef @ dPt)) / Pn
        total = 0.0
        for dag, exc, Phi, sgn, R in sides:
            dPhi = start_vectors(exc, words, dcoef, n, orbitals, dag)
            dHs = H.build(um, exc).dense()
            dA = sgn * dE0 * np.eye(len(exc)) - sgn * dHs
            for iz in range(len(z)):
                Rz = R[iz]
                RPhi = Rz @ Phi
                dG = dPhi.T @ RPhi + RPhi.T @ dPhi - RPhi.T @ dA @ RPhi
                total += float(np.sum(np.real(np.conj(gc[iz]) * dG)))
        kind, i, j = par
        if kind == "t":
            gt[i, j] = gt[j, i] = total
        elif kind == "eps":
            ge[i] = total
        else:
            gu[i] = total
    return gt, ge, gu
