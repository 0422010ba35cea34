"""Impurity models for the batched workload: a 2x2 open plaquette (t = 1)
coupled to 8 bath sites, one instance per seed.

Inputs only (shared by the oracle tests and the library's tests and
benchmark); nothing of the method's arithmetic.

Instance k (numpy PCG64 seeded with 1000 + k):
  sites 0..3   cluster, bonds (0,1), (1,3), (3,2), (2,0) with t_ij = -1,
               U ~ uniform[2, 8] (one value for the four sites), eps = -U/2;
  sites 4..11  bath, eps_b ~ uniform[-2, 2], U = 0, hybridised with every
               cluster site: t_ib ~ normal(0, 0.5^2);
  half filling N_up = N_dn = 6; Monte Carlo basis size N_f log-uniform in
  [1e3, 1e5]; sampling temperature U beta = 1.6 (the paper's rule for other U).
Seed state: at half filling with up and down electrons on complementary sites
every double-occupancy-free state has the same diagonal energy (sum of all
eps); the one of smallest word is taken: up on sites 0..5, down on 6..11.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

N_CLUSTER = 4
N_BATH = 8
N_SITES = N_CLUSTER + N_BATH
PLAQUETTE = [(0, 1), (1, 3), (3, 2), (2, 0)]


@dataclass
class Impurity:
    k: int
    t: np.ndarray          # [12, 12] symmetric
    eps: np.ndarray        # [12]
    U_sites: np.ndarray    # [12]
    U: float
    n_f: int
    beta: float
    n_up: int = 6
    n_dn: int = 6
    seed: int = 0

    @property
    def n_sites(self) -> int:
        return N_SITES

    def seed_word(self) -> int:
        up = (1 << 6) - 1
        dn = ((1 << N_SITES) - 1) ^ up
        return (up << N_SITES) | dn

    def bath_params(self):
        """(eps_bath [8], hybridisation [4, 8]) as stored in eps and t."""
        return self.eps[N_CLUSTER:].copy(), self.t[:N_CLUSTER, N_CLUSTER:].copy()


def impurity(k: int, n_f: int | None = None) -> Impurity:
    rng = np.random.Generator(np.random.PCG64(1000 + k))
    U = float(rng.uniform(2.0, 8.0))
    eps_bath = rng.uniform(-2.0, 2.0, N_BATH)
    hyb = rng.normal(0.0, 0.5, (N_CLUSTER, N_BATH))
    nf = int(round(10 ** rng.uniform(3.0, 5.0))) if n_f is None else int(n_f)
    t = np.zeros((N_SITES, N_SITES))
    for i, j in PLAQUETTE:
        t[i, j] = t[j, i] = -1.0
    t[:N_CLUSTER, N_CLUSTER:] = hyb
    t[N_CLUSTER:, :N_CLUSTER] = hyb.T
    eps = np.concatenate([np.full(N_CLUSTER, -U / 2), eps_bath])
    Us = np.concatenate([np.full(N_CLUSTER, U), np.zeros(N_BATH)])
    return Impurity(k, t, eps, Us, U, nf, 1.6 / U, seed=k)


def batch(n: int, n_f: int | None = None) -> list[Impurity]:
    return [impurity(k, n_f) for k in range(n)]
