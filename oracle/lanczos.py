"""Ground state of H~: the Lanczos recursion of App. B and dense diagonalisation.

App. B builds a Krylov basis from a random start vector phi_0 with

    phi_{n+1} = H phi_n - a_n phi_n - b_n^2 phi_{n-1},
    a_n   = <phi_n|H|phi_n> / <phi_n|phi_n>,
    b_n^2 = <phi_n|phi_n> / <phi_{n-1}|phi_{n-1}>,   b_0 = 0, phi_{-1} = 0,

and diagonalises the tridiagonal matrix with a_n on the diagonal and b_n
(n >= 1) beside it.  Two readings (the printed text is garbled there):
the recursion's last coefficient is b_n^2, since with the unnormalised vectors
that the a_n, b_n^2 definitions use only b_n^2 makes phi_{n+1} orthogonal to
phi_{n-1}; and the normalised basis vectors are |n> = phi_n / sqrt(<phi_n|phi_n>).
The ground state in the truncated basis is sum_n |n> <n|Omega_eff> (the
change-of-basis Eq. of App. B).

No reorthogonalisation (the paper uses none).  The unnormalised vectors grow
like prod b_n; when |phi_n| leaves [1e-100, 1e100] both phi_n and phi_{n-1}
are rescaled by the same factor, which leaves every a_n and b_n^2 unchanged.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class LanczosResult:
    E0: float
    a: np.ndarray
    b: np.ndarray            # b[0] = 0, b[n] for n >= 1
    iters: int
    psi: np.ndarray | None   # normalised ground state in the basis, if asked for
    residual: float          # |H psi - E0 psi| when psi is formed, else estimate


def start_vector(n: int, seed: int) -> np.ndarray:
    """A random start vector (App. B only asks for "a random initial vector")."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def tridiag_ground(a: np.ndarray, b: np.ndarray):
    """Lowest eigenpair of the tridiagonal H_eff (a on the diagonal, b[1:] beside)."""
    m = len(a)
    if m == 1:
        return float(a[0]), np.ones(1)
    w, V = sla.eigh_tridiagonal(a, b[1:m], select="i", select_range=(0, 0))
    return float(w[0]), V[:, 0]


def lanczos(apply, n: int, max_iter: int = 400, tol: float = 1e-12, seed: int = 0,
            phi0: np.ndarray | None = None, want_vector: bool = False) -> LanczosResult:
    """Run App. B's recursion with the matrix-vector product ``apply``.

    Stops when the Ritz residual estimate b_{m} |s_{m-1}| (the last component of
    the tridiagonal ground-state eigenvector times the next b) falls below
    ``tol`` * max(1, |E0|), when b_{n+1} vanishes (invariant subspace), or
    after ``max_iter`` steps.
    """
    phi = start_vector(n, seed) if phi0 is None else np.array(phi0, dtype=np.float64)
    phi_prev = np.zeros(n)
    nn_prev = 1.0
    a, b = [], []
    vecs = [] if want_vector else None
    E0, s = 0.0, None
    resid_est = np.inf
    for it in range(max_iter):
        nn = float(phi @ phi)
        if it > 0 and nn <= (1e-14 * max(1.0, abs(E0))) ** 2 * nn_prev:
            break                                  # invariant subspace reached
        if nn > 1e200 or nn < 1e-200:              # joint rescale, leaves a_n, b_n^2 unchanged
            f = 1.0 / np.sqrt(nn)
            phi, phi_prev, nn_prev, nn = phi * f, phi_prev * f, nn_prev * f * f, 1.0
        Hphi = apply(phi)
        an = float(phi @ Hphi) / nn
        b2 = nn / nn_prev if it > 0 else 0.0
        a.append(an)
        b.append(np.sqrt(b2))
        if want_vector:
            vecs.append(phi / np.sqrt(nn))
        phi_next = Hphi - an * phi - b2 * phi_prev
        E0, s = tridiag_ground(np.array(a), np.array(b))
        bnext = np.sqrt(float(phi_next @ phi_next) / nn)
        resid_est = abs(bnext * s[-1])
        phi_prev, phi, nn_prev = phi, phi_next, nn
        if resid_est < tol * max(1.0, abs(E0)):
            break
    a, b = np.array(a), np.array(b)
    psi = None
    residual = resid_est
    if want_vector:
        psi = np.zeros(n)
        for c, v in zip(s, vecs):
            psi += c * v
        psi /= np.linalg.norm(psi)
        residual = float(np.linalg.norm(apply(psi) - E0 * psi))
    return LanczosResult(E0, a, b, len(a), psi, residual)


def dense_ground(H: np.ndarray):
    """Lowest eigenpair by dense symmetric diagonalisation (library eigh)."""
    w, V = np.linalg.eigh(H)
    return float(w[0]), V[:, 0], w
