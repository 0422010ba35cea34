"""Seeded, synthetic inputs shared by the oracle and the CUDA path.

Holds lattices (hopping matrices), named workload configurations and seeded
random vectors.  It contains none of the method's arithmetic (no hops, signs,
lookups, sampling or Krylov steps).
"""
from . import lattice, configs  # noqa: F401
from .vectors import random_block  # noqa: F401
