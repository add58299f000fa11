"""SplitMix64 counter stream and checkerboard cell phases (oracle side).

Test infrastructure only (see ``oracle/__init__``).

The paper (Sec. 2, Eq. 3) draws each cell of the L^3 lattice independently:
``a_m(x) = lambda + beta * ahat_m(x)`` with ``ahat`` in {0, 1} per cell, so a
cell is either the low value ``lambda`` or the high value ``lambda + beta``.
The paper names no generator. We fix one: the SplitMix64 stream of
Steele, Lea & Flood ("Fast splittable pseudorandom number generators",
OOPSLA 2014). The i-th output (i = 0, 1, ...) of the stream seeded with
``seed`` is ``mix64(seed + (i + 1) * GAMMA)`` mod 2^64, where ``mix64`` is the
published finalizer (two xor-shift-multiply rounds and a final xor-shift).

Cell ``(c1, c2, c3)`` takes output number ``c3 + L*c2 + L^2*c1`` (the paper's
big-endian index with x3 fastest, Sec. 3.2) and is high iff the top 53 bits of
that output, read as an integer u, satisfy ``u < floor(p_hi * 2^53)``.
For p_hi = 1/2 this is "top bit clear".

Pinned by the published SplitMix64 test vectors (tests/golden/splitmix64.txt)
and by the binomial count of high cells.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX_M1 = 0xBF58476D1CE4E5B9
MIX_M2 = 0x94D049BB133111EB


def mix64(z: int) -> int:
    """SplitMix64 output finalizer on a Python int (mod 2^64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX_M1) & MASK64
    z = ((z ^ (z >> 27)) * MIX_M2) & MASK64
    return z ^ (z >> 31)


def splitmix64_outputs(seed: int, count: int) -> list[int]:
    """First ``count`` outputs of the SplitMix64 stream seeded with ``seed``.

    Written as the sequential generator: advance the state by GAMMA, then mix.
    """
    state = seed & MASK64
    out = []
    for _ in range(count):
        state = (state + GAMMA) & MASK64
        out.append(mix64(state))
    return out


def splitmix64_at(seed: int, index: int) -> int:
    """Output number ``index`` of the stream, by direct (counter) evaluation."""
    return mix64((seed + (index + 1) * GAMMA) & MASK64)


def hi_threshold(p_hi: float) -> int:
    """Integer threshold on the top 53 bits: floor(p_hi * 2^53) (exact in FP64)."""
    if not (0.0 <= p_hi <= 1.0):
        raise ValueError("p_hi must lie in [0, 1]")
    return int(p_hi * 9007199254740992.0)


def cell_phases(L: int, seed: int, p_hi: float = 0.5) -> np.ndarray:
    """Phase (1 = high value, 0 = low value) of every cell, shape (L, L, L).

    Pure-Python integer loop: the obviously correct version, used for L <= 16.
    """
    thr = hi_threshold(p_hi)
    ph = np.zeros((L, L, L), dtype=np.uint8)
    for c1 in range(L):
        for c2 in range(L):
            for c3 in range(L):
                u = splitmix64_at(seed, c3 + L * c2 + L * L * c1) >> 11
                ph[c1, c2, c3] = 1 if u < thr else 0
    return ph


def cell_phases_vec(L: int, seed: int, p_hi: float = 0.5) -> np.ndarray:
    """Same as :func:`cell_phases`, vectorised with numpy uint64 (wraps mod 2^64).

    Checked against the loop version in the tests; used for large L.
    """
    thr = np.uint64(hi_threshold(p_hi))
    idx = np.arange(L * L * L, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX_M2)
        z = z ^ (z >> np.uint64(31))
    u = z >> np.uint64(11)
    return (u < thr).astype(np.uint8).reshape(L, L, L)


def cell_values(phase: np.ndarray, a_lo: float, a_hi: float) -> np.ndarray:
    """Cell coefficient a = a_lo on low cells, a_hi on high cells (Eq. 3 with
    a_lo = lambda, a_hi = lambda + beta)."""
    return np.where(phase.astype(bool), float(a_hi), float(a_lo))


# ---------------------------------------------------------------- contrast levels
# Varying contrast (Sec. 2, the two-contrast and layer-type realizations): a
# cell takes one of K levels 0 .. K-1 with the coefficient values[level]. The
# draw uses the same output u (top 53 bits) as the two-level rule: with the
# tail probabilities P_m = probs[m] + probs[m+1] + ... + probs[K-1], summed in
# FP64 from the top level down, and T_m = floor(P_m * 2^53), the level is the
# number of m in 1 .. K-1 with u < T_m. For K = 2 (probs = (1 - p_hi, p_hi))
# T_1 = floor(p_hi * 2^53): the two-level rule above.


def level_thresholds(probs) -> list[int]:
    """Integer thresholds T_1 >= ... >= T_{K-1} of the level draw."""
    K = len(probs)
    if K < 2 or any(not (0.0 <= float(p) <= 1.0) for p in probs):
        raise ValueError("need K >= 2 probabilities in [0, 1]")
    tail = 0.0
    T = [0] * K
    for m in range(K - 1, 0, -1):
        tail = float(probs[m]) + tail
        T[m] = int(min(tail, 1.0) * 9007199254740992.0)
    return T[1:]


def cell_levels(L: int, seed: int, probs) -> np.ndarray:
    """Level (0 .. K-1) of every cell, shape (L, L, L); pure-Python loop."""
    T = level_thresholds(probs)
    lv = np.zeros((L, L, L), dtype=np.uint8)
    for c1 in range(L):
        for c2 in range(L):
            for c3 in range(L):
                u = splitmix64_at(seed, c3 + L * c2 + L * L * c1) >> 11
                lv[c1, c2, c3] = sum(1 for t in T if u < t)
    return lv


def cell_levels_vec(L: int, seed: int, probs) -> np.ndarray:
    """Same as :func:`cell_levels`, vectorised (checked against it in the tests)."""
    T = level_thresholds(probs)
    idx = np.arange(L * L * L, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX_M2)
        z = z ^ (z >> np.uint64(31))
    u = z >> np.uint64(11)
    lv = np.zeros(L * L * L, dtype=np.uint8)
    for t in T:
        lv += (u < np.uint64(t)).astype(np.uint8)
    return lv.reshape(L, L, L)


def level_values(level: np.ndarray, values) -> np.ndarray:
    """Cell coefficient values[min(level, K-1)] (a level byte past the top
    level reads as the top level)."""
    v = np.asarray(values, dtype=np.float64)
    return v[np.minimum(level.astype(np.int64), len(v) - 1)]
