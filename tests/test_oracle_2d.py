"""Pins for the 2D oracle (the paper's 2D experiments, Sec. 5): the
x3-invariant 3D scheme, Keller duality against the independent voxel scheme,
the checkerboard product, the laminate, Fourier eigenvalues and a
manufactured solution."""
import numpy as np
import pytest

from oracle import assembly, dual2d, homogenized, pcg, precond, rng, solver2d


def test_2d_draw_is_the_first_slab_of_the_3d_draw():
    for L, seed, p in ((4, 0, 0.5), (6, 11, 0.3), (5, 2**63 + 1, 0.8)):
        assert np.array_equal(solver2d.cell_phases_2d(L, seed, p), rng.cell_phases(L, seed, p)[0])
        assert np.array_equal(solver2d.cell_phases_2d_vec(L, seed, p), solver2d.cell_phases_2d(L, seed, p))
    assert np.array_equal(solver2d.cell_phases_2d_vec(40, 9, 0.5), rng.cell_phases_vec(40, 9, 0.5)[0])


@pytest.mark.parametrize("sub", [None, 2])
def test_equals_the_x3_invariant_3d_scheme(sub):
    # the 3D edge coefficient of an x3-invariant field is the mean of four
    # voxels, two of which repeat the other two: the 2D mean of two
    L, n = 4, 4
    ph = solver2d.cell_phases_2d(L, 3)
    V2 = solver2d.voxel_field_2d(ph, n, 1.0, 10.0, sub)
    a2 = solver2d.edge_coefficients_2d(V2)
    N = L * n
    V3 = np.repeat(V2[:, :, None], N, axis=2)
    a3 = assembly.edge_coefficients_voxels(V3)
    for d in range(2):
        assert np.array_equal(a3[d][:, :, 0], a2[d])
    psis2, _, H2, _ = solver2d.solve_2d(V2)
    A3 = assembly.stiffness_edges(a3)
    psis3 = [pcg.tight_solve(A3, assembly.rhs(a3, i), N)[0].reshape(N, N, N) for i in range(2)] + [None]
    H3 = homogenized.ahom_edge(a3, psis3)
    assert np.abs(H3[:2, :2] - H2).max() <= 1e-10


def test_keller_duality_and_checkerboard_product():
    # sigma and 1/sigma: A[sigma] R A_vox[1/sigma] R^T = I (independent voxel scheme)
    ph = solver2d.cell_phases_2d(4, 9)
    V = solver2d.voxel_field_2d(ph, 2, 1.0, 7.0)
    _, _, H, _ = solver2d.solve_2d(V)
    Hv = dual2d.ahom_voxel_2d(1.0 / V)
    Rm = np.array([[0.0, -1.0], [1.0, 0.0]])
    assert np.allclose(H @ Rm @ Hv @ Rm.T, np.eye(2), atol=1e-10)
    # two-phase checkerboard: A_node A_vox = alpha beta, sqrt(alpha beta) between
    al, be = 1.0, 10.0
    V = np.repeat(np.repeat(np.array([[al, be], [be, al]]), 4, 0), 4, 1)
    _, _, H, _ = solver2d.solve_2d(V)
    Hv = dual2d.ahom_voxel_2d(V)
    assert abs(H[0, 0] * Hv[0, 0] - al * be) <= 1e-9 * al * be
    assert Hv[0, 0] < np.sqrt(al * be) < H[0, 0]


@pytest.mark.parametrize("axis", [0, 1])
def test_laminate_closed_form(axis):
    vals = np.array([1.0, 5.0, 2.0, 9.0])
    n = 3
    col = np.repeat(vals, n)
    V = np.broadcast_to(col[:, None] if axis == 0 else col[None, :], (col.size, col.size)).copy()
    psis, _, H, a = solver2d.solve_2d(V)
    want = np.full(2, vals.mean())
    want[axis] = 1.0 / np.mean(1.0 / vals)
    assert np.abs(np.diag(H) - want).max() <= 1e-11
    assert abs(H[0, 1]) <= 1e-11 and abs(H[1, 0]) <= 1e-11
    assert np.abs(solver2d.ahom_2d_energy(a, psis) - H).max() <= 1e-10


def test_constant_coefficient_fourier_eigenvalues():
    N, c = 12, 3.5
    A = solver2d.stiffness_2d(solver2d.edge_coefficients_2d(np.full((N, N), c)))
    lam = precond.laplacian_eigenvalues(N)
    j = np.arange(N)
    for k1, k2 in ((0, 1), (3, 5), (6, 6), (11, 2)):
        v = np.cos(2 * np.pi * (k1 * j[:, None] + k2 * j[None, :]) / N).ravel()
        assert np.abs(A @ v - c * (lam[k1] + lam[k2]) * v).max() <= 1e-12
    assert np.abs(np.asarray(A.sum(axis=1)).ravel()).max() <= 1e-13
    assert abs(A - A.T).max() <= 1e-15


def test_manufactured_solution_and_preconditioners():
    N = 16
    V = solver2d.voxel_field_2d(solver2d.cell_phases_2d(4, 1), 4, 1.0, 100.0)
    a = solver2d.edge_coefficients_2d(V)
    A = solver2d.stiffness_2d(a)
    j = np.arange(N)
    psi = np.sin(2 * np.pi * j / N)[:, None] * np.cos(4 * np.pi * j / N)[None, :]
    b = A @ psi.ravel()
    for G in (solver2d.core_2d_exact(N), solver2d.core_2d_from_nodes(N, *precond.rank_r_nodes(N, 8))):
        x, it, rel = pcg.pcg(A, b, lambda r: solver2d.apply_precond_2d(G, r.reshape(N, N)).ravel(), tol=1e-13)
        assert np.abs(x - psi.ravel()).max() <= 1e-10
    # the exact preconditioner is the pseudo-inverse of the constant-coefficient operator
    L1 = solver2d.stiffness_2d(solver2d.edge_coefficients_2d(np.ones((N, N))))
    r = np.random.default_rng(0).standard_normal(N * N)
    r -= r.mean()
    z = solver2d.apply_precond_2d(solver2d.core_2d_exact(N), r.reshape(N, N)).ravel()
    assert np.abs(L1 @ z - r).max() <= 1e-12
