"""Pins for the oracle's SplitMix64 stream and checkerboard cell phases."""
import math
import os

import numpy as np
import pytest

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            s, i, v = line.split()
            rows.append((int(s), int(i), int(v)))
    return rows


def test_splitmix64_published_vectors():
    rows = _golden()
    assert len(rows) >= 8
    for seed, idx, val in rows:
        assert rng.splitmix64_outputs(seed, idx + 1)[idx] == val
        assert rng.splitmix64_at(seed, idx) == val


def test_counter_form_equals_sequential():
    for seed in (0, 1, 7, 2**63 + 5, 2**64 - 1):
        seq = rng.splitmix64_outputs(seed, 50)
        assert seq == [rng.splitmix64_at(seed, i) for i in range(50)]


@pytest.mark.parametrize("L,seed,p", [(4, 0, 0.5), (5, 3, 0.5), (6, 11, 0.3), (3, 2**40 + 1, 0.9)])
def test_vectorised_phases_match_loop(L, seed, p):
    assert np.array_equal(rng.cell_phases(L, seed, p), rng.cell_phases_vec(L, seed, p))


def test_phase_definition_top_bit():
    # p = 1/2: high iff the top bit of the output is clear
    L, seed = 4, 9
    ph = rng.cell_phases(L, seed)
    for c in range(L ** 3):
        top = rng.splitmix64_at(seed, c) >> 63
        assert ph.ravel()[c] == (1 - top)


def test_extreme_probabilities():
    assert rng.cell_phases_vec(6, 1, 0.0).sum() == 0
    assert rng.cell_phases_vec(6, 1, 1.0).sum() == 216


def test_high_count_binomial():
    # paper: about L^3/2 inclusions (Sec. 2; Table 3 column S, e.g. 16338 of 32768 at L=32)
    for seed in range(4):
        L = 32
        k = int(rng.cell_phases_vec(L, seed).sum())
        mu, sd = L ** 3 / 2, math.sqrt(L ** 3) / 2
        assert abs(k - mu) < 5 * sd


def test_cell_values():
    ph = np.array([[[0, 1], [1, 0]], [[1, 1], [0, 0]]], dtype=np.uint8)
    v = rng.cell_values(ph, 1.0, 100.0)
    assert v[0, 0, 1] == 100.0 and v[0, 0, 0] == 1.0
