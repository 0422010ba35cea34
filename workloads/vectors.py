"""Seeded random input vectors for H*v parity tests and benchmarks."""
from __future__ import annotations

import numpy as np


def random_block(n: int, ncols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """[n, ncols] row-major block of N(0, 1) entries from numpy's PCG64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, ncols)).astype(dtype)
