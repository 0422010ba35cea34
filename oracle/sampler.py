"""Monte Carlo construction of the truncated basis F~ (Sec. "Subspace of the
ground state").

What the paper fixes:
* start from one very probable state (an antiferromagnetic state);
* propose new states by applying every hopping term of the kinetic part;
* accept a proposed state b with probability min(exp(-U beta n_U(b)), 1)
  (the Boltzmann-factor Eq.), which depends on the proposed state only;
* proceed by steps: the states accepted in one step are the starting points of
  the next; already-accepted states may be proposed again ("revisited") and do
  not grow F~;
* stop when F~ holds N_f states; F~ is kept as a searchable set.

What the paper leaves open, and the reading taken here (both this oracle and
the library's sampler follow it, each written independently):
* random numbers: one SplitMix64 draw per proposal, keyed by
  (seed, step, parent word, hop id) -- see ``draw``;
* acceptance: u = (draw >> 11) * 2^-53 < exp(-beta * sum_i U_i n_i,up n_i,dn)
  (this is the paper's factor for uniform U, written per site);
* hop id of c^dag_{i s} c_{j s}: s * n^2 + i * n + j (s = 0 up, 1 down);
  every ordered pair with t_ij != 0 is a hopping term;
* next starting points: every state accepted in the step, new or already in
  F~ ("revisit" reading); flag NEW_ONLY keeps only the new ones;
* a step that would overshoot N_f adds only the N_f - |F~| new states of
  smallest priority ``prio(seed, word)`` (ties by word), so |F~| = N_f exactly
  and bases of one seed are nested in N_f;
* the run also stops when a step accepts nothing or after 64 consecutive
  steps without a new state (then fewer than N_f states are returned).

Parity of this module against the paper is unpinned (the paper's generator and
seeds are not published); it is pinned to SplitMix64's published outputs, to
acceptance statistics and to structural invariants.
"""
from __future__ import annotations

import math

import numpy as np

from . import fock

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
C1 = 0xBF58476D1CE4E5B9
C2 = 0x94D049BB133111EB
NEW_ONLY = 1
STAGNATION_STEPS = 64


# --- SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; Vigna's splitmix64.c) ------
def mix64_int(z: int) -> int:
    """SplitMix64 output function on a Python int."""
    z &= M64
    z = ((z ^ (z >> 30)) * C1) & M64
    z = ((z ^ (z >> 27)) * C2) & M64
    return z ^ (z >> 31)


def splitmix64_stream(state: int, count: int) -> list[int]:
    """The generator's output sequence: state += golden gamma; emit mix64(state)."""
    out = []
    for _ in range(count):
        state = (state + GOLDEN) & M64
        out.append(mix64_int(state))
    return out


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function, vectorised over uint64 arrays (wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(C1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(C2)
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int) -> int:
    return mix64_int((seed + GOLDEN) & M64)


def draw(seed: int, step: int, parents: np.ndarray, hop: int) -> np.ndarray:
    """64-bit draw for proposals (seed, step, parent, hop):
    mix64(mix64(mix64(key(seed) ^ step) ^ parent) ^ hop)."""
    k2 = mix64_int(stream_key(seed) ^ (step & M64))
    k3 = mix64(np.uint64(k2) ^ np.asarray(parents, dtype=np.uint64))
    return mix64(k3 ^ np.uint64(hop))


def prio(seed: int, words: np.ndarray) -> np.ndarray:
    """Truncation priority: the draw of step 2^64 - 1 (never a real step)."""
    k2 = mix64_int(stream_key(seed) ^ M64)
    return mix64(np.uint64(k2) ^ np.asarray(words, dtype=np.uint64))


def acceptance(words: np.ndarray, n: int, U: np.ndarray, beta: float) -> np.ndarray:
    """min(exp(-beta * sum_i U_i n_i,up n_i,dn), 1) per word (Boltzmann-factor Eq.).

    exp is evaluated by Python's math.exp once per distinct interaction energy.
    """
    up, dn = fock.split(words, n)
    both = up & dn
    EU = np.zeros(len(both))
    for i in range(n):
        EU += U[i] * ((both >> np.uint64(i)) & np.uint64(1)).astype(np.float64)
    vals, inv = np.unique(EU, return_inverse=True)
    p = np.array([min(math.exp(-beta * v), 1.0) for v in vals])
    return p[inv]


def proposals(frontier: np.ndarray, n: int, t: np.ndarray):
    """Every (parent, hop id, child) obtained by one hopping term on a frontier word."""
    up, dn = fock.split(frontier, n)
    one = np.uint64(1)
    for spin, ws, shift in ((0, up, n), (1, dn, 0)):
        for i, j, _ in fock.directed_hops(t):
            ok = (((ws >> np.uint64(j)) & one) == one) & (((ws >> np.uint64(i)) & one) == 0)
            if not ok.any():
                continue
            par = frontier[ok]
            child = par ^ np.uint64(((1 << i) | (1 << j)) << shift)
            yield par, spin * n * n + i * n + j, child


def sample_basis(n: int, t: np.ndarray, U: np.ndarray, n_up: int, n_dn: int,
                 n_target: int, beta: float, seeds, seed: int = 0, flags: int = 0,
                 max_steps: int = 1 << 20, trace: list | None = None) -> np.ndarray:
    """Grow F~ step by step until it holds n_target states; returns sorted words."""
    F = np.unique(np.asarray(seeds, dtype=np.uint64))
    up, dn = fock.split(F, n)
    if np.any(fock.popcount(up) != n_up) or np.any(fock.popcount(dn) != n_dn):
        raise ValueError("seed state outside the (N_up, N_dn) sector")
    if len(F) > n_target:
        raise ValueError("more seed states than n_target")
    frontier = F
    step = 0
    stagnant = 0
    while len(F) < n_target and step < max_steps:
        step += 1
        acc = []
        for par, hop, child in proposals(frontier, n, t):
            u = (draw(seed, step, par, hop) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
            keep = u < acceptance(child, n, U, beta)
            acc.append(child[keep])
        accepted = np.unique(np.concatenate(acc)) if acc else np.zeros(0, np.uint64)
        new = np.setdiff1d(accepted, F, assume_unique=True)
        room = n_target - len(F)
        if len(new) > room:
            order = np.lexsort((new, prio(seed, new)))
            new = np.sort(new[order[:room]])
        F = np.union1d(F, new).astype(np.uint64)
        if trace is not None:
            trace.append((step, len(frontier), len(accepted), len(new), len(F)))
        frontier = new if (flags & NEW_ONLY) else accepted
        stagnant = stagnant + 1 if len(new) == 0 else 0
        if len(accepted) == 0 or len(frontier) == 0 or stagnant >= STAGNATION_STEPS:
            break
    return F
