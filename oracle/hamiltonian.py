"""The projected Hamiltonian H~_mn = <x~_m|H|x~_n> on a set of basis words.

Eq. (1) of the paper with t_ij, eps_i, U_i, restricted to the truncated basis
F~ (the Eq. defining the truncated-basis matrix in Sec. "Subspace of the
ground state").  App. B states that discarding the Fock states an application
of H produces outside F~ is the same as applying this projected matrix; the
oracle therefore builds the matrix explicitly: every hop of every basis state
is enumerated and kept only when its target is in the basis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import fock


@dataclass
class Model:
    n: int
    t: np.ndarray
    eps: np.ndarray
    U: np.ndarray


@dataclass
class Projected:
    """H~ in coordinate form: off-diagonal entries (row, col, value) + diagonal."""
    basis: np.ndarray      # sorted uint64 words
    rows: np.ndarray       # int64, target index  (H~[row, col] = <row|H|col>)
    cols: np.ndarray       # int64, source index
    vals: np.ndarray       # float64, t_ij * sign
    diag: np.ndarray       # float64

    @property
    def n(self) -> int:
        return len(self.basis)

    def dense(self) -> np.ndarray:
        H = np.zeros((self.n, self.n))
        H[self.rows, self.cols] += self.vals
        H[np.arange(self.n), np.arange(self.n)] += self.diag
        return H

    def sparse(self):
        import scipy.sparse as sp
        off = sp.coo_matrix((self.vals, (self.rows, self.cols)), shape=(self.n, self.n))
        return (off + sp.diags(self.diag)).tocsr()

    def nnz_offdiag(self) -> int:
        return int(len(self.vals))


def build(model: Model, basis) -> Projected:
    """Enumerate c^dag_{i s} c_{j s} on every basis word; keep in-basis targets.

    Vectorised over basis states for each directed hop (i, j, spin); the
    target's position is found with a sorted search (a library primitive).
    """
    basis = np.asarray(basis, dtype=np.uint64)
    n = model.n
    N = len(basis)
    up, dn = fock.split(basis, n)
    rows, cols, vals = [], [], []
    one = np.uint64(1)
    for spin, ws, shift in ((0, up, n), (1, dn, 0)):
        for i, j, tij in fock.directed_hops(model.t):
            elig = (((ws >> np.uint64(j)) & one) == one) & (((ws >> np.uint64(i)) & one) == 0)
            src = np.nonzero(elig)[0]
            if len(src) == 0:
                continue
            flip = np.uint64(((1 << i) | (1 << j)) << shift)
            tgt = basis[src] ^ flip
            nb = fock.popcount(ws[src] & np.uint64(fock.between_mask(i, j)))
            sign = np.where(nb % 2 == 0, 1.0, -1.0)
            pos = np.searchsorted(basis, tgt)
            ok = pos < N
            ok[ok] &= basis[pos[ok]] == tgt[ok]
            rows.append(pos[ok].astype(np.int64))
            cols.append(src[ok].astype(np.int64))
            vals.append(tij * sign[ok])
    if rows:
        r, c, v = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    else:
        r = c = np.zeros(0, np.int64)
        v = np.zeros(0)
    order = np.lexsort((c, r))
    d = fock.diagonal(basis, n, model.eps, model.U)
    return Projected(basis, r[order], c[order], v[order], d)


def apply_exact(P: Projected, x: np.ndarray) -> np.ndarray:
    """y = H~ x with every row summed by math.fsum (correctly rounded).

    x may be [N] or [N, L]; the result is independent of summation order.
    Pure Python per row: use on small bases only.
    """
    x = np.asarray(x, dtype=np.float64)
    X = x.reshape(P.n, -1)
    Y = np.zeros_like(X)
    starts = np.searchsorted(P.rows, np.arange(P.n + 1))
    for r in range(P.n):
        a, b = starts[r], starts[r + 1]
        cs, vs = P.cols[a:b], P.vals[a:b]
        for col in range(X.shape[1]):
            terms = [P.diag[r] * X[r, col]] + [float(v) * X[c, col] for c, v in zip(cs, vs)]
            Y[r, col] = math.fsum(terms)
    return Y.reshape(x.shape)


def apply_abs(P: Projected, x: np.ndarray) -> np.ndarray:
    """|H~| |x| row sums, the scale of the rounding-error bound of y = H~ x."""
    A = P.sparse()
    A.data = np.abs(A.data)
    X = np.abs(np.asarray(x, dtype=np.float64)).reshape(P.n, -1)
    return (A @ X).reshape(np.shape(x))


def row(model: Model, basis: np.ndarray, k: int):
    """Row k of H~ from scratch: (cols, vals, diag), by hopping state k itself.

    H~ is real symmetric, so <x_k|H|x_c> equals the amplitude of the hop that
    takes x_k to x_c.  Used to check sampled rows at sizes where the full
    matrix is too large to build.
    """
    n = model.n
    w = int(basis[k])
    cols, vals = [], []
    for spin in (0, 1):
        for i, j, tij in fock.directed_hops(model.t):
            h = fock.hop_word(w, n, spin, i, j)
            if h is None:
                continue
            w2, s = h
            p = int(np.searchsorted(basis, np.uint64(w2)))
            if p < len(basis) and int(basis[p]) == w2:
                cols.append(p)
                vals.append(tij * s)
    d = float(fock.diagonal(np.array([w], dtype=np.uint64), n, model.eps, model.U)[0])
    return np.array(cols, dtype=np.int64), np.array(vals), d


def apply_rows(model: Model, basis: np.ndarray, x: np.ndarray, ks) -> tuple[np.ndarray, np.ndarray]:
    """(y[ks], (|H~||x|)[ks]) evaluated row by row with math.fsum."""
    X = np.asarray(x, dtype=np.float64).reshape(len(basis), -1)
    Y = np.zeros((len(ks), X.shape[1]))
    S = np.zeros_like(Y)
    for a, k in enumerate(ks):
        cs, vs, d = row(model, basis, int(k))
        for col in range(X.shape[1]):
            terms = [d * X[k, col]] + [v * X[c, col] for c, v in zip(cs, vs)]
            Y[a, col] = math.fsum(terms)
            S[a, col] = math.fsum(abs(t) for t in terms)
    return Y, S


def parameter_derivatives(model: Model, basis, u: np.ndarray, v: np.ndarray):
    """d<u, H~ v>/d(t_ij, eps_i, U_i) from the plain definition: H~ is linear
    in its parameters, so each derivative is <u, D v> with D the projected
    Hamiltonian of that parameter alone set to 1 (for t_ij: the bond (i, j)
    with t_ij = t_ji = 1).  Returns (grad_t [n, n] symmetric, 0 off the bonds,
    grad_eps [n], grad_U [n]); u, v are [N] or [N, L] (summed over columns)."""
    n = model.n
    U_ = np.asarray(u, dtype=np.float64).reshape(len(basis), -1)
    V_ = np.asarray(v, dtype=np.float64).reshape(len(basis), -1)
    zero = np.zeros(n)
    gt = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if model.t[i, j] == 0.0:
                continue
            T = np.zeros((n, n))
            T[i, j] = T[j, i] = 1.0
            D = build(Model(n, T, zero, zero), basis).sparse()
            gt[i, j] = gt[j, i] = float(np.sum(U_ * (D @ V_)))
    ge = np.zeros(n)
    gu = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        de = fock.diagonal(np.asarray(basis, dtype=np.uint64), n, e, zero)
        du = fock.diagonal(np.asarray(basis, dtype=np.uint64), n, zero, e)
        ge[i] = float(np.sum(U_ * (de[:, None] * V_)))
        gu[i] = float(np.sum(U_ * (du[:, None] * V_)))
    return gt, ge, gu
