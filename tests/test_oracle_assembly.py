"""Pins for the oracle's stiffness matrix, edge coefficients and RHS.

What pins them (not the oracle's own formulas):
* the paper's Kronecker sum over cells (Sec. 3.3, Eq. 18) and the edge form
  are two different constructions that must give the same matrix;
* symmetry and A 1 = 0 (periodic Neumann structure, Sec. 3.2);
* for a constant coefficient c, A = c A_Delta acts on each Fourier mode with
  the closed-form eigenvalue c (l1 + l2 + l3), l = 4 sin^2(pi k / N)
  (Sec. 4.2, Eqs. 27-29);
* the nodal weights 1, 1/2, 1/4 of Sec. 3.3 (Fig. 4) on a single inclusion;
* the RHS sums to zero and vanishes for a constant coefficient.
"""
import numpy as np
import pytest

from oracle import assembly, rng


def _cells(L, seed, lo=1.0, hi=10.0):
    return rng.cell_values(rng.cell_phases(L, seed), lo, hi)


@pytest.mark.parametrize("L,n,seed", [(2, 2, 0), (3, 2, 1), (2, 4, 5), (4, 2, 7), (3, 3, 2)])
def test_kron_cell_sum_equals_edge_form(L, n, seed):
    cv = _cells(L, seed)
    A1 = assembly.stiffness_kron_cells(cv, n)
    A2 = assembly.stiffness_edges(assembly.edge_coefficients(cv, n))
    assert abs(A1 - A2).max() < 1e-13


@pytest.mark.parametrize("L,n,seed", [(3, 2, 3), (4, 4, 0)])
def test_symmetric_and_zero_row_sums(L, n, seed):
    A = assembly.stiffness_edges(assembly.edge_coefficients(_cells(L, seed), n))
    assert abs(A - A.T).max() == 0.0
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-12
    # positive semidefinite with a one-dimensional kernel (tiny grid, dense check)
    if A.shape[0] <= 512:
        ev = np.linalg.eigvalsh(A.toarray())
        assert ev[0] > -1e-10 and ev[1] > 1e-8


def test_constant_coefficient_fourier_modes():
    N, c = 8, 3.5
    cv = np.full((4, 4, 4), c)
    A = assembly.stiffness_edges(assembly.edge_coefficients(cv, 2))
    j = np.arange(N)
    for m in [(0, 0, 1), (1, 2, 3), (4, 0, 2), (3, 3, 3)]:
        phase = 2 * np.pi * (m[0] * j[:, None, None] + m[1] * j[None, :, None] + m[2] * j[None, None, :]) / N
        for mode in (np.cos(phase), np.sin(phase)):
            lam = sum(4 * np.sin(np.pi * mk / N) ** 2 for mk in m)
            assert np.allclose(A @ mode.ravel(), c * lam * mode.ravel(), atol=1e-12)


def test_nodal_weights_single_inclusion():
    # one high cell (value 1) in a zero background: edge coefficients are
    # 1 inside, 1/2 on the faces of the inclusion, 1/4 on its edges (Sec. 3.3)
    L, n = 3, 4
    cv = np.zeros((L, L, L))
    cv[1, 1, 1] = 1.0
    a = assembly.edge_coefficients(cv, n)
    lo, hi = n, 2 * n  # nodes of the inclusion along each axis
    # x1-edges starting at j1 in [lo, hi) run inside the inclusion along x1
    assert a[0][lo, lo + 1, lo + 1] == 1.0        # interior
    assert a[0][lo, lo, lo + 1] == 0.5            # on a face (j2 on the boundary)
    assert a[0][lo, lo, lo] == 0.25               # on an edge (j2, j3 on the boundary)
    assert a[0][lo, hi, hi] == 0.25
    assert a[0][lo - 1, lo + 1, lo + 1] == 0.0    # outside along x1
    assert a[0][hi, lo + 1, lo + 1] == 0.0
    # total: each voxel shares 4 edges per axis with weight 1/4 -> mean = volume fraction
    for d in range(3):
        assert abs(a[d].mean() - 1 / L ** 3) < 1e-15


def test_matrix_free_stencil_matches_csr():
    cv = _cells(4, 3, 1.0, 100.0)
    a = assembly.edge_coefficients(cv, 3)
    A = assembly.stiffness_edges(a)
    psi = np.random.default_rng(0).standard_normal(a.shape[1:])
    assert np.allclose(assembly.apply_stencil(a, psi).ravel(), A @ psi.ravel(), rtol=0, atol=1e-11)


def test_rhs_properties():
    cv = _cells(4, 1)
    a = assembly.edge_coefficients(cv, 4)
    for i in range(3):
        b = assembly.rhs(a, i)
        assert abs(b.sum()) < 1e-12
        # b_i(j) = a_i(j) - a_i(j - e_i)
        assert np.allclose(b.reshape(a.shape[1:]), a[i] - np.roll(a[i], 1, axis=i), atol=0)
    ac = assembly.edge_coefficients(np.full((2, 2, 2), 7.0), 3)
    assert np.abs(assembly.rhs(ac, 0)).max() == 0.0


def test_point_evaluators_match_full_arrays():
    cv = _cells(4, 3, 1.0, 100.0)
    n = 3
    a = assembly.edge_coefficients(cv, n)
    psi = np.random.default_rng(5).standard_normal(a.shape[1:])
    Ap = assembly.apply_stencil(a, psi)
    rng_ = np.random.default_rng(6)
    for _ in range(40):
        j = tuple(int(v) for v in rng_.integers(0, 12, 3))
        assert abs(assembly.apply_at(cv, n, lambda k: psi[k], j) - Ap[j]) < 1e-12
        for i in range(3):
            assert abs(assembly.rhs_at(cv, n, i, j) - assembly.rhs(a, i).reshape(a.shape[1:])[j]) < 1e-14
            assert assembly.edge_coefficient_at(cv, n, i, j) == a[i][j]
