"""Pins for sub-cell inclusions (Sec. 3.1: a centred cube of side 2 alpha n
grid intervals per unit cell carries the random coefficient, the rest is
lambda = a_lo)."""
import numpy as np
import pytest

from oracle import assembly, homogenized, pcg, problem, rng


def test_full_sub_cell_is_the_checkerboard():
    ph = rng.cell_phases(3, 5)
    V = assembly.inclusion_field(ph, 4, 4, 1.0, 10.0)
    assert np.array_equal(V, assembly.voxel_field(rng.cell_values(ph, 1.0, 10.0), 4))
    a = problem.realization(3, 4, 5, 1.0, 10.0, sub=4).a_edges
    assert np.array_equal(a, problem.realization(3, 4, 5, 1.0, 10.0).a_edges)


def test_inclusion_geometry_and_volume():
    # one high cell, n = 8, sub = 4: exactly the voxels 2..5 of that cell on each axis
    ph = np.zeros((2, 2, 2), dtype=np.uint8)
    ph[1, 0, 1] = 1
    V = assembly.inclusion_field(ph, 8, 4, 0.4, 1.0)
    hi = np.argwhere(V == 1.0)
    assert hi.shape[0] == 4 ** 3
    assert hi[:, 0].min() == 8 + 2 and hi[:, 0].max() == 8 + 5
    assert hi[:, 1].min() == 2 and hi[:, 1].max() == 5
    assert hi[:, 2].min() == 8 + 2 and hi[:, 2].max() == 8 + 5
    # mean coefficient = a_lo + (a_hi - a_lo) * f_cells * (sub/n)^3 for any phases
    ph = rng.cell_phases(4, 9)
    V = assembly.inclusion_field(ph, 8, 4, 0.4, 1.0)
    assert abs(V.mean() - (0.4 + 0.6 * ph.mean() / 8.0)) < 1e-14


def test_invalid_sub_cell():
    for sub in (0, 9, 3):
        with pytest.raises(ValueError):
            assembly.inclusion_field(np.zeros((2, 2, 2), dtype=np.uint8), 8, sub, 1.0, 2.0)


def test_periodic_array_of_cubes_is_isotropic():
    # every cell high: a cubic lattice of cubes, symmetric under axis
    # permutations and reflections, so A_hom = a I exactly (Sec. 3.4 edge form)
    re = problem.realization(2, 4, 0, 1.0, 10.0, p_hi=1.0, sub=2)
    psis = [pcg.tight_solve(re.A, re.b[i], re.N)[0].reshape(re.N, re.N, re.N) for i in range(3)]
    A = homogenized.ahom_edge(re.a_edges, psis)
    off = A - np.diag(np.diag(A))
    assert np.abs(off).max() < 1e-10
    assert np.abs(np.diag(A) - A[0, 0]).max() < 1e-10
    # between a_lo and the arithmetic mean of the edge coefficients
    assert 1.0 < A[0, 0] < re.a_edges[0].mean()
