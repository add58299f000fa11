"""Seeded synthetic inputs shared by the tests (no arithmetic of the method).

Random fields are plain seeded draws; the coefficient realizations themselves
are generated from (L, n, seed, p_hi, a_lo, a_hi) by each side independently.
"""
from __future__ import annotations

import numpy as np


def random_field(N: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard-normal N^3 field, shape (N, N, N)."""
    return np.random.default_rng(seed).standard_normal((N, N, N)).astype(dtype)


def sample_nodes(N: int, count: int, seed: int):
    """Distinct grid nodes, always including the corners of the periodic box."""
    rng = np.random.default_rng(seed)
    nodes = {(0, 0, 0), (N - 1, N - 1, N - 1), (0, N - 1, 0), (N - 1, 0, N - 1)}
    while len(nodes) < count:
        nodes.add(tuple(int(v) for v in rng.integers(0, N, 3)))
    return sorted(nodes)
