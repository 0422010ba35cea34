"""Fock states as 64-bit words, symmetry sectors and single-hop matrix elements.

Encoding (App. D: |90> = |0101;1010> has the spin-up occupations in the high
half): word = (up << n) | dn, bit i of each half = site i.  Fermionic modes are
ordered "all up modes 0..n-1, then all down modes 0..n-1" (Jordan-Wigner).

Hopping c^dag_{i s} c_{j s} on an occupation word w_s of spin s (i != j, bit j
set, bit i clear) moves one electron past the occupied same-spin modes lying
strictly between i and j, so its matrix element is
(-1)^(number of occupied same-spin sites strictly between i and j).
"""
from __future__ import annotations

from itertools import combinations

import numpy as np

_POP16 = np.array([bin(i).count("1") for i in range(1 << 16)], dtype=np.int64)


def popcount(x) -> np.ndarray:
    """Number of set bits of each uint64 entry (table lookup, 16 bits at a time)."""
    x = np.asarray(x, dtype=np.uint64)
    m = np.uint64(0xFFFF)
    return (_POP16[(x & m).astype(np.int64)]
            + _POP16[((x >> np.uint64(16)) & m).astype(np.int64)]
            + _POP16[((x >> np.uint64(32)) & m).astype(np.int64)]
            + _POP16[((x >> np.uint64(48)) & m).astype(np.int64)])


def words_with_popcount(n: int, k: int) -> list[int]:
    """All n-bit integers with exactly k set bits, ascending."""
    out = []
    for sites in combinations(range(n), k):
        w = 0
        for s in sites:
            w |= 1 << s
        out.append(w)
    out.sort()
    return out


def sector(n: int, n_up: int, n_dn: int) -> np.ndarray:
    """Every word of the (N_up, N_dn) sector, ascending (Sec. ED: the block with
    N_e electrons and spin S_z has C(n, N_up) * C(n, N_dn) states)."""
    ups = np.array(words_with_popcount(n, n_up), dtype=np.uint64)
    dns = np.array(words_with_popcount(n, n_dn), dtype=np.uint64)
    return ((ups[:, None] << np.uint64(n)) | dns[None, :]).reshape(-1)


def split(words: np.ndarray, n: int) -> tuple[np.ndarray, np.ndarray]:
    w = np.asarray(words, dtype=np.uint64)
    mask = np.uint64((1 << n) - 1)
    return w >> np.uint64(n), w & mask


def between_mask(i: int, j: int) -> int:
    """Bits strictly between sites i and j."""
    lo, hi = min(i, j), max(i, j)
    return ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)


def directed_hops(t: np.ndarray) -> list[tuple[int, int, float]]:
    """(i, j, t_ij) for every ordered pair i != j with t_ij != 0."""
    n = t.shape[0]
    return [(i, j, float(t[i, j])) for i in range(n) for j in range(n)
            if i != j and t[i, j] != 0.0]


def hop_word(w: int, n: int, spin: int, i: int, j: int):
    """Apply c^dag_{i,spin} c_{j,spin} to word w.

    Returns (new_word, sign) or None if the hop is not allowed.  spin 0 = up
    (high half), 1 = down (low half).
    """
    shift = n if spin == 0 else 0
    ws = (w >> shift) & ((1 << n) - 1)
    if not (ws >> j) & 1 or (ws >> i) & 1:
        return None
    nb = bin(ws & between_mask(i, j)).count("1")
    return w ^ (((1 << i) | (1 << j)) << shift), (-1) ** nb


def double_occupancy(words, n: int) -> np.ndarray:
    """n_U = number of doubly occupied sites (Sec. ED, definition of n_U)."""
    up, dn = split(words, n)
    return popcount(up & dn)


def diagonal(words, n: int, eps: np.ndarray, U: np.ndarray) -> np.ndarray:
    """<w|H|w> = sum_i eps_i (n_i,up + n_i,dn) + sum_i U_i n_i,up n_i,dn (Eq. (1))."""
    up, dn = split(words, n)
    d = np.zeros(len(up), dtype=np.float64)
    one = np.uint64(1)
    for i in range(n):
        ui = ((up >> np.uint64(i)) & one).astype(np.float64)
        di = ((dn >> np.uint64(i)) & one).astype(np.float64)
        d += eps[i] * (ui + di) + U[i] * (ui * di)
    return d


def annihilate(w: int, n: int, n_up: int, spin: int, i: int):
    """c_{i,spin}|w> -> (new_word, sign) or None (mode order: up modes, then down)."""
    shift = n if spin == 0 else 0
    ws = (w >> shift) & ((1 << n) - 1)
    if not (ws >> i) & 1:
        return None
    before = bin(ws & ((1 << i) - 1)).count("1")
    if spin == 1:
        before += bin(w >> n).count("1")
    return w ^ (1 << (i + shift)), (-1) ** before


def create(w: int, n: int, spin: int, i: int):
    """c^dag_{i,spin}|w> -> (new_word, sign) or None."""
    shift = n if spin == 0 else 0
    ws = (w >> shift) & ((1 << n) - 1)
    if (ws >> i) & 1:
        return None
    before = bin(ws & ((1 << i) - 1)).count("1")
    if spin == 1:
        before += bin(w >> n).count("1")
    return w | (1 << (i + shift)), (-1) ** before
