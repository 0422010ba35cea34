"""Named workloads: the clusters, fillings and Monte Carlo settings.

Each entry is a plain description (lattice, U, eps, filling, basis size,
sampling temperature, seed).  The paper fixes t = 1, U = 8, beta = 0.2 and,
for other U, U*beta = 1.6 (Sec. "Results" and "1D Lattice, variable U").
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lattice as L


@dataclass
class Workload:
    name: str
    lat: L.Lattice
    U: float
    n_up: int
    n_dn: int
    n_f: int                 # Monte Carlo basis size target
    beta: float              # Monte Carlo inverse temperature (U*beta = 1.6)
    seed: int = 0
    mu: float = 0.0          # eps_i = -mu

    @property
    def n_sites(self) -> int:
        return self.lat.n_sites

    @property
    def eps(self) -> np.ndarray:
        return np.full(self.lat.n_sites, -self.mu)

    @property
    def U_sites(self) -> np.ndarray:
        return np.full(self.lat.n_sites, self.U)

    def seed_word(self) -> int:
        return L.afm_seed(self.lat, self.n_up, self.n_dn)


def ring8_u4() -> Workload:
    """8-site periodic ring, U = 4, N_up = N_dn = 4, 2000 MC states, seed 0."""
    return Workload("ring8_U4_nf2000", L.ring(8), 4.0, 4, 4, 2000, 1.6 / 4.0)


def tilted12_u8() -> Workload:
    """12-site tilted cluster R=((4,0),(1,3)), U = 8, 6+6 electrons, 2^18 states."""
    return Workload("tilted12_U8_nf262144", L.superlattice_cluster((4, 0), (1, 3)),
                    8.0, 6, 6, 1 << 18, 0.2)


def square16_u8() -> Workload:
    """4x4 periodic, t' = -0.3, U = 8, 7+7 electrons, 1e7 MC states."""
    return Workload("square4x4_tp-0.3_U8_nf1e7",
                    L.superlattice_cluster((4, 0), (0, 4), t=1.0, tp=-0.3),
                    8.0, 7, 7, 10_000_000, 0.2)


def rect24_u8() -> Workload:
    """6x4 periodic, t' = -0.3, U = 8, 11+11 electrons, 5e7 MC states."""
    return Workload("rect6x4_tp-0.3_U8_nf5e7",
                    L.superlattice_cluster((6, 0), (0, 4), t=1.0, tp=-0.3),
                    8.0, 11, 11, 50_000_000, 0.2)


WORKLOADS = {
    "ring8": ring8_u4,
    "tilted12": tilted12_u8,
    "square16": square16_u8,
    "rect24": rect24_u8,
}
