"""Pins for multi-level coefficients (varying contrast, Sec. 2: inclusion
cells carry lambda + beta_c with a contrast beta_c drawn per cell, or set per
layer of cells; the background is lambda)."""
import numpy as np
import pytest

from oracle import assembly, homogenized, pcg, problem, rng


@pytest.mark.parametrize("probs", [(0.2, 0.5, 0.3), (0.5, 0.0, 0.5), (0.1, 0.2, 0.3, 0.4), (0.0, 0.0, 1.0)])
def test_level_draw_loop_matches_vectorised(probs):
    for seed in (0, 7, 2**63 + 5):
        assert np.array_equal(rng.cell_levels(5, seed, probs), rng.cell_levels_vec(5, seed, probs))


@pytest.mark.parametrize("p_hi", [0.0, 0.25, 0.5, 0.7, 1.0])
def test_two_levels_are_the_checkerboard_draw(p_hi):
    # K = 2 with probs (1 - p_hi, p_hi) is the two-level rule, bit for bit
    for seed in (3, 11):
        assert np.array_equal(rng.cell_levels(4, seed, (1.0 - p_hi, p_hi)), rng.cell_phases(4, seed, p_hi))
        assert np.array_equal(rng.cell_levels_vec(20, seed, (1.0 - p_hi, p_hi)), rng.cell_phases_vec(20, seed, p_hi))


def test_level_frequencies_are_multinomial():
    probs = (0.2, 0.5, 0.3)
    lv = rng.cell_levels_vec(32, 1234, probs)
    n = lv.size
    for k, p in enumerate(probs):
        cnt = int((lv == k).sum())
        assert abs(cnt - n * p) < 5.0 * np.sqrt(n * p * (1 - p))
    # nested events: level >= m iff u < T_m, so raising the top level's share
    # only promotes cells (never demotes one)
    lv2 = rng.cell_levels_vec(32, 1234, (0.2, 0.3, 0.5))
    assert np.all(lv2 >= np.minimum(lv, 1)) and np.all(lv2[lv == 2] == 2)


def test_thresholds_and_invalid_probabilities():
    assert rng.level_thresholds((0.5, 0.5)) == [2**52]
    assert rng.level_thresholds((0.0, 0.25, 0.75)) == [2**53, 3 * 2**51]
    with pytest.raises(ValueError):
        rng.level_thresholds((1.0,))
    with pytest.raises(ValueError):
        rng.level_thresholds((0.5, -0.1, 0.6))


def test_level_field_two_levels_is_inclusion_field():
    ph = rng.cell_phases(3, 5)
    for sub in (8, 4, 2):
        V = assembly.level_field(ph, 8, (0.4, 1.0), sub)
        assert np.array_equal(V, assembly.inclusion_field(ph, 8, sub, 0.4, 1.0))


def test_level_field_geometry_and_clamp():
    lv = np.zeros((2, 2, 2), dtype=np.uint8)
    lv[1, 0, 1] = 2
    lv[0, 1, 0] = 1
    lv[1, 1, 1] = 7  # past the top level: reads as level K - 1
    V = assembly.level_field(lv, 4, (0.4, 0.7, 1.0), sub=2)
    assert np.array_equal(np.argwhere(V == 0.7)[:, 0], np.full(8, 1) + np.repeat([0, 1], 4))
    assert (V == 1.0).sum() == 16 and (V == 0.7).sum() == 8
    assert V[4 + 1, 0 + 1, 4 + 2] == 1.0 and V[0, 0, 0] == 0.4
    # relabelling the levels together with their values leaves the field unchanged
    perm = np.array([0, 2, 1], dtype=np.uint8)
    V2 = assembly.level_field(perm[np.minimum(lv, 2)], 4, (0.4, 1.0, 0.7), sub=2)
    assert np.array_equal(V, V2)


def test_operator_is_linear_in_the_level_values():
    # the edge coefficients are means of voxel values, so the stiffness is
    # sum_l v_l A(indicator of level l)
    lv = rng.cell_levels(2, 9, (0.3, 0.3, 0.4))
    vals = (0.4, 0.7, 1.3)
    A = problem.realization_levels(2, 4, 0, vals, level=lv, sub=2).A
    parts = [problem.realization_levels(2, 4, 0, tuple(1.0 if k == m else 0.0 for k in range(3)), level=lv, sub=2).A
             for m in range(3)]
    S = sum(v * P for v, P in zip(vals, parts))
    assert abs(A - S).max() < 1e-14


def test_single_level_medium_is_homogeneous():
    # every cell at level 2 with whole-cell inclusions: a = values[2]
    # everywhere, b = 0, psi = 0 and A_hom = values[2] I
    lv = np.full((3, 3, 3), 2, dtype=np.uint8)
    re = problem.realization_levels(3, 2, 0, (0.4, 0.7, 1.0), level=lv)
    assert max(np.abs(b).max() for b in re.b) == 0.0
    A = homogenized.ahom_edge(re.a_edges, [np.zeros((6, 6, 6))] * 3)
    assert np.array_equal(A, np.diag([1.0, 1.0, 1.0]))


@pytest.mark.parametrize("axis", [0, 2])
def test_three_level_laminate_closed_form(axis):
    # layer-type medium: the level depends on one cell coordinate only. The
    # corrector along that axis makes the flux constant, so A_aa is the
    # harmonic mean of the cell values over the layers and the other two
    # diagonal entries are arithmetic means; the off-diagonal entries vanish.
    L, n = 6, 2
    vals = np.array([0.4, 0.7, 1.0])
    layer = np.array([0, 2, 1, 1, 2, 0], dtype=np.uint8)
    shape = [1, 1, 1]
    shape[axis] = L
    lv = np.broadcast_to(layer.reshape(shape), (L, L, L)).copy()
    re = problem.realization_levels(L, n, 0, vals, level=lv)
    psis = [pcg.tight_solve(re.A, re.b[i], re.N)[0].reshape(re.N, re.N, re.N) for i in range(3)]
    A = homogenized.ahom_edge(re.a_edges, psis)
    v = vals[layer]
    harm, arith = 1.0 / np.mean(1.0 / v), np.mean(v)
    want = np.full(3, arith)
    want[axis] = harm
    assert np.abs(np.diag(A) - want).max() < 1e-10
    assert np.abs(A - np.diag(np.diag(A))).max() < 1e-10


def test_random_three_level_edge_bounds():
    # harmonic mean of a_i over the x_i-edges <= A_ii <= their arithmetic mean
    # (Cauchy-Schwarz on the flux, and the zero corrector as a competitor)
    re = problem.realization_levels(3, 4, 21, (0.4, 0.7, 1.0), probs=(0.5, 0.25, 0.25), sub=2)
    psis = [pcg.tight_solve(re.A, re.b[i], re.N)[0].reshape(re.N, re.N, re.N) for i in range(3)]
    A = homogenized.ahom_edge(re.a_edges, psis)
    E = homogenized.ahom_energy(re.a_edges, psis)
    assert np.abs(A - E).max() < 1e-9 and np.abs(A - A.T).max() < 1e-9
    for i in range(3):
        ai = re.a_edges[i]
        assert 1.0 / np.mean(1.0 / ai) - 1e-12 <= A[i, i] <= ai.mean() + 1e-12
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() >= 0.4 and ev.max() <= 1.0
