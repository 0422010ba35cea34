"""Cluster geometry -> Hubbard parameters (t_ij, eps_i, U_i).

This module only builds *inputs*: the hopping matrix of a periodic cluster,
the on-site energies and the site coordinates used to pick an
antiferromagnetic seed state.  It holds none of the method's arithmetic and is
shared by the oracle and by the CUDA path's tests and benchmark.

Model: Eq. (1) of the paper, H = -t sum c^dag c + U sum n_up n_dn - mu sum n,
generalised to a real symmetric hopping matrix t_ij (i != j), on-site energies
eps_i (eps_i = -mu for the paper's model) and on-site repulsions U_i.

Periodic clusters (Sec. "Results", 2D superlattice vectors in the caption of
Fig. 5): the sites are the integer points of one cell of the superlattice
spanned by R1 = (a, 0), R2 = (b, c); site index = y * a + x for 0 <= x < a,
0 <= y < c.  Hoppings are accumulated per displacement vector, so a bond that
wraps onto an already-connected pair is counted again (a "multigraph"): this
is the reading that reproduces the paper's 2x4 full-ED energy (Table of 2D
energies, N_c = 8).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Lattice:
    """A cluster: hopping matrix, site coordinates and a two-colouring."""

    name: str
    n_sites: int
    t: np.ndarray                 # [n, n] real symmetric, zero diagonal
    coords: np.ndarray            # [n, 2] integer site coordinates
    sublattice: np.ndarray        # [n] 0 = A, 1 = B ((x + y) even -> A)
    notes: dict = field(default_factory=dict)


def _reduce(x: int, y: int, a: int, b: int, c: int) -> tuple[int, int]:
    """Bring (x, y) into the cell 0 <= x < a, 0 <= y < c of R1=(a,0), R2=(b,c)."""
    k = y // c
    x -= k * b
    y -= k * c
    x %= a
    return x, y


def superlattice_cluster(R1, R2, t: float = 1.0, tp: float = 0.0,
                         name: str | None = None) -> Lattice:
    """Square-lattice cluster with periodic superlattice vectors R1, R2.

    R1 must be (a, 0) and R2 = (b, c) with a, c > 0 (upper-triangular form);
    every square-lattice cluster of the paper and of the benchmark configs has
    this form.  Nearest-neighbour amplitude t enters as t_ij = -t, the
    next-nearest-neighbour amplitude t' as t_ij = -t' (the usual t-t' sign
    convention; t' is not in the paper).
    """
    a, r1y = R1
    b, c = R2
    if r1y != 0 or a <= 0 or c <= 0:
        raise ValueError("superlattice vectors must be R1=(a,0), R2=(b,c) with a,c>0")
    n = a * c
    coords = np.array([(x, y) for y in range(c) for x in range(a)], dtype=np.int64)
    index = {(int(x), int(y)): i for i, (x, y) in enumerate(coords)}
    T = np.zeros((n, n), dtype=np.float64)
    shells = [((1, 0), (0, 1)), ((1, 1), (1, -1))]
    amps = [-t, -tp]
    for disp, amp in zip(shells, amps):
        if amp == 0.0:
            continue
        for i, (x, y) in enumerate(coords):
            for dx, dy in disp:
                j = index[_reduce(int(x) + dx, int(y) + dy, a, b, c)]
                if j == i:
                    continue
                T[i, j] += amp
                T[j, i] += amp
    sub = (coords[:, 0] + coords[:, 1]) % 2
    return Lattice(name or f"R=(({a},0),({b},{c}))", n, T, coords, sub.astype(np.int64),
                   {"R1": (a, 0), "R2": (b, c), "t": t, "tp": tp})


def ring(n: int, t: float = 1.0, name: str | None = None) -> Lattice:
    """Periodic 1D ring; each nearest-neighbour bond is added once per site."""
    T = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        j = (i + 1) % n
        if j == i:
            continue
        T[i, j] += -t
        T[j, i] += -t
    coords = np.array([(i, 0) for i in range(n)], dtype=np.int64)
    return Lattice(name or f"ring{n}", n, T, coords, (np.arange(n) % 2).astype(np.int64),
                   {"t": t})


def dimer(t: float = 1.0) -> Lattice:
    """Two sites joined by a single bond t_01 = -t (not a 2-site ring)."""
    T = np.array([[0.0, -t], [-t, 0.0]])
    return Lattice("dimer", 2, T, np.array([(0, 0), (1, 0)]), np.array([0, 1]), {"t": t})


def afm_seed(lat: Lattice, n_up: int, n_dn: int) -> int:
    """Antiferromagnetic seed word (Sec. "Subspace of the ground state").

    Up electrons go on the lowest-index A sites, down electrons on the
    lowest-index B sites; at half filling this fills both sublattices (the
    paper's |90> = |0101;1010> on the 4-site ring).  If a sublattice has fewer
    sites than electrons the remaining electrons take the lowest free sites of
    the other sublattice.  The word layout is (up << n_sites) | dn, bit i of
    each half = site i.
    """
    n = lat.n_sites
    A = [i for i in range(n) if lat.sublattice[i] == 0]
    B = [i for i in range(n) if lat.sublattice[i] == 1]

    def fill(pref, other, k):
        sites = pref[:k]
        if len(sites) < k:
            sites += [s for s in other if s not in sites][: k - len(sites)]
        return sites

    up = 0
    for s in fill(A, B, n_up):
        up |= 1 << s
    dn = 0
    for s in fill(B, A, n_dn):
        dn |= 1 << s
    return (up << n) | dn
