"""The 2D solver (the paper's 2D experiments, Sec. 5) through the C ABI
against the 2D oracle: cells, operator, RHS, preconditioner (up to N = 2048),
solves and A_hom (up to N = 512), closed forms and argument checks."""
import functools

import numpy as np
import pytest

from oracle import dual2d, pcg, precond, rng, solver2d
from tests import inputs

pytestmark = pytest.mark.gpu

# the oracle's exponential sum fitted on the 2D spectrum: the expected G of the
# rank-R tests, never the library's factors
_oracle_nodes_2d = functools.lru_cache(maxsize=None)(lambda N, R: precond.lsq_nodes(N, R, 2))


@pytest.fixture(scope="module")
def sq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2007_06524_gb300 as pkg

    return pkg


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _field2d(N, seed):
    return np.random.default_rng(seed).standard_normal((N, N))


@pytest.mark.parametrize("L,seed,p", [(4, 0, 0.5), (6, 3, 0.3), (64, 7, 0.5), (32, 2**63 + 5, 0.9)])
def test_cells_bit_exact(sq, L, seed, p):
    c = sq.sq2d_build_coeffs(L, 4, seed, p, 1.0, 10.0)
    got = sq.sq2d_coeffs_cells(c)
    want = solver2d.cell_phases_2d(L, seed, p) if L <= 6 else solver2d.cell_phases_2d_vec(L, seed, p)
    assert np.array_equal(got, want)


def test_cells_bit_exact_sampled_at_l512(sq):
    L, seed = 512, 5
    got = sq.sq2d_coeffs_cells(sq.sq2d_build_coeffs(L, 4, seed, 0.5, 1.0, 10.0))
    r = np.random.default_rng(1)
    thr = rng.hi_threshold(0.5)
    for c1, c2 in r.integers(0, L, size=(400, 2)):
        want = 1 if (rng.splitmix64_at(seed, int(c2) + L * int(c1)) >> 11) < thr else 0
        assert got[c1, c2] == want


GRIDS = [(2, 4, None), (4, 4, 2), (3, 4, 2), (6, 8, 4), (12, 8, None), (64, 4, 2), (96, 4, 2), (256, 4, 2),
         (512, 4, 2)]


@pytest.mark.parametrize("L,n,sub", GRIDS)
def test_operator_and_rhs(sq, L, n, sub):
    import torch

    N = L * n
    ph = solver2d.cell_phases_2d(L, 11) if L <= 16 else solver2d.cell_phases_2d_vec(L, 11)
    c = sq.sq2d_coeffs_from_host(L, n, ph.ravel(), 0.4, 1.0)
    if sub is not None:
        sq.sq2d_coeffs_set_subcell(c, sub)
    a = solver2d.edge_coefficients_2d(solver2d.voxel_field_2d(ph, n, 0.4, 1.0, sub))
    A = solver2d.stiffness_2d(a)
    x = _field2d(N, N)
    y = torch.empty(N * N, dtype=torch.float64, device="cuda")
    sq.sq2d_apply_operator(c, _dev(x.ravel()), y)
    ref = A @ x.ravel()
    assert _relmax(y.cpu().numpy(), ref) <= 1e-13
    for i in range(2):
        sq.sq2d_rhs(c, i, y)
        assert np.abs(y.cpu().numpy() - solver2d.rhs_2d(a, i)).max() <= 1e-15


@pytest.mark.parametrize("N", [8, 12, 16, 48, 96, 256, 384, 1024, 2048])
@pytest.mark.parametrize("rank", [0, 4, 8])
def test_preconditioner(sq, N, rank):
    import torch

    pc = sq.sq2d_precond_setup(N, rank)
    w = sq.sq2d_workspace_create(N)
    r = _field2d(N, 3 * N + rank)
    z = torch.empty(N * N, dtype=torch.float64, device="cuda")
    sq.sq2d_apply_precond(pc, w, _dev(r.ravel()), z)
    G = solver2d.core_2d_exact(N) if rank == 0 else solver2d.core_2d_from_nodes(N, *_oracle_nodes_2d(N, rank))
    ref = solver2d.apply_precond_2d(G, r)
    # both sides round in their transforms at about eps log N relative to the
    # input, while the output's max is set by the lowest modes (G ~ N^2 / 4 pi^2):
    # the max-norm relative difference grows with N
    assert _relmax(z.cpu().numpy().reshape(N, N), ref) <= 1e-12 * max(1.0, N / 256)


@pytest.mark.parametrize("N,R", [(256, 8), (16, 4), (2048, 8), (96, 6)])
def test_rank_r_fit_matches_oracle_on_the_2d_spectrum(sq, N, R):
    """The 2D exponential sum (fitted on {l_i + l_j}) against the oracle's
    independent construction on the same spectrum."""
    t, w = sq.sq2d_precond_factors(sq.sq2d_precond_setup(N, R), R)
    to, wo = _oracle_nodes_2d(N, R)
    assert np.all(w > 0) and np.abs(t / to - 1).max() <= 1e-13
    x = precond.spectrum_values(N, 2)
    g, go = np.exp(-np.outer(x, t)) @ w, np.exp(-np.outer(x, to)) @ wo
    assert np.abs(g / go - 1).max() <= 1e-12


@pytest.mark.parametrize("L,n,sub,rank", [(4, 4, 2, 0), (8, 4, 2, 8), (16, 4, None, 4), (32, 4, 2, 8), (64, 4, 2, 0),
                                          (128, 4, 2, 8)])
def test_solves_and_ahom(sq, L, n, sub, rank):
    import torch

    N = L * n
    ph = solver2d.cell_phases_2d(L, 21) if L <= 16 else solver2d.cell_phases_2d_vec(L, 21)
    c = sq.sq2d_build_coeffs(L, n, 21, 0.5, 0.4, 1.0)
    assert np.array_equal(sq.sq2d_coeffs_cells(c), ph)
    if sub is not None:
        sq.sq2d_coeffs_set_subcell(c, sub)
    V = solver2d.voxel_field_2d(ph, n, 0.4, 1.0, sub)
    psis_o, _, Ho, a = solver2d.solve_2d(V, tol=1e-13)
    pc = sq.sq2d_precond_setup(N, rank)
    w = sq.sq2d_workspace_create(N)
    psis = []
    for i in range(2):
        psi = torch.empty(N * N, dtype=torch.float64, device="cuda")
        info = sq.sq2d_pcg_solve(c, pc, w, i, 1e-12, 4000, psi)
        assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-12
        x = psi.cpu().numpy().reshape(N, N)
        assert np.linalg.norm(x - psis_o[i]) / np.linalg.norm(psis_o[i]) <= 1e-9
        psis.append(psi)
    H, E = sq.sq2d_homogenized_matrix(c, *psis)
    assert np.abs(H - Ho).max() <= 1e-10 * np.abs(Ho).max()
    assert np.abs(E - Ho).max() <= 1e-9 * np.abs(Ho).max()


@pytest.mark.parametrize("axis", [0, 1])
def test_laminate_closed_form(sq, axis):
    import torch

    L, n = 8, 4
    N = L * n
    layer = np.array([0, 1, 1, 0, 1, 0, 0, 1], dtype=np.uint8)
    ph = np.broadcast_to(layer[:, None] if axis == 0 else layer[None, :], (L, L)).copy()
    c = sq.sq2d_coeffs_from_host(L, n, ph.ravel(), 1.0, 6.0)
    pc = sq.sq2d_precond_setup(N, 0)
    w = sq.sq2d_workspace_create(N)
    psis = [torch.empty(N * N, dtype=torch.float64, device="cuda") for _ in range(2)]
    for i in range(2):
        assert sq.sq2d_pcg_solve(c, pc, w, i, 1e-13, 2000, psis[i])["status"] == sq.SQ_OK
    H, E = sq.sq2d_homogenized_matrix(c, *psis)
    v = np.where(layer > 0, 6.0, 1.0)
    want = np.full(2, v.mean())
    want[axis] = 1.0 / np.mean(1.0 / v)
    assert np.abs(np.diag(H) - want).max() <= 1e-11 and abs(H[0, 1]) <= 1e-11


def test_checkerboard_duality_with_the_voxel_scheme(sq):
    """Two-phase checkerboard: A_node (GPU) x A_vox (independent oracle voxel
    scheme) = alpha beta, with sqrt(alpha beta) strictly between."""
    import torch

    al, be, n = 1.0, 10.0, 8
    ph = np.array([[0, 1], [1, 0]], dtype=np.uint8)
    c = sq.sq2d_coeffs_from_host(2, n, ph.ravel(), al, be)
    N = 2 * n
    pc = sq.sq2d_precond_setup(N, 0)
    w = sq.sq2d_workspace_create(N)
    psis = [torch.empty(N * N, dtype=torch.float64, device="cuda") for _ in range(2)]
    for i in range(2):
        sq.sq2d_pcg_solve(c, pc, w, i, 1e-13, 2000, psis[i])
    H, _ = sq.sq2d_homogenized_matrix(c, *psis)
    Hv = dual2d.ahom_voxel_2d(solver2d.voxel_field_2d(ph, n, al, be))
    assert abs(H[0, 0] * Hv[0, 0] - al * be) <= 1e-9 * al * be
    assert Hv[0, 0] < np.sqrt(al * be) < H[0, 0]


def test_paper_setting_l512_properties(sq):
    """The paper's largest 2D case: L = 512, n0 = 4, alpha = 1/4 (N = 2048,
    4.2 M unknowns), rank-8 preconditioner, tol 1e-8: both correctors meet the
    recomputed FP64 residual, A_hom is symmetric with equal edge and energy
    forms, and each diagonal entry lies between the harmonic and arithmetic
    means of its edge coefficients."""
    import torch

    L, n = 512, 4
    N = L * n
    c = sq.sq2d_build_coeffs(L, n, 3, 0.5, 0.4, 1.0)
    sq.sq2d_coeffs_set_subcell(c, 2)
    pc = sq.sq2d_precond_setup(N, 8)
    w = sq.sq2d_workspace_create(N)
    psis = [torch.empty(N * N, dtype=torch.float64, device="cuda") for _ in range(2)]
    for i in range(2):
        info = sq.sq2d_pcg_solve(c, pc, w, i, 1e-8, 3000, psis[i])
        assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-8
    H, E = sq.sq2d_homogenized_matrix(c, *psis)
    assert abs(H[0, 1] - H[1, 0]) <= 1e-7 and np.abs(H - E).max() <= 1e-7
    ph = sq.sq2d_coeffs_cells(c)
    a = solver2d.edge_coefficients_2d(solver2d.voxel_field_2d(ph, n, 0.4, 1.0, 2))
    for i in range(2):
        assert 1.0 / np.mean(1.0 / a[i]) - 1e-9 <= H[i, i] <= a[i].mean() + 1e-9


def test_invalid_arguments(sq):
    import torch

    for L, n in ((1024, 4), (5, 2), (3, 3)):  # N = 4096, 10, 9
        with pytest.raises(sq.SqError):
            sq.sq2d_build_coeffs(L, n, 0, 0.5, 1.0, 2.0)
    with pytest.raises(sq.SqError):
        sq.sq2d_precond_setup(4096, 0)
    c = sq.sq2d_build_coeffs(8, 4, 0, 0.5, 1.0, 2.0)
    with pytest.raises(sq.SqError):
        sq.sq2d_coeffs_set_subcell(c, 3)
    pc, w = sq.sq2d_precond_setup(64, 0), sq.sq2d_workspace_create(32)
    psi = torch.empty(32 * 32, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SqError):
        sq.sq2d_pcg_solve(c, pc, w, 0, 1e-8, 100, psi)  # N mismatch
    with pytest.raises(sq.SqError):
        sq.sq2d_pcg_solve(c, sq.sq2d_precond_setup(32, 0), w, 2, 1e-8, 100, psi)


def test_iteration_graphs_match_direct_launches_2d(sq):
    """2D solves replay a CUDA graph of two iterations (SQ_OPT_PCG_GRAPHS = 1)
    or launch every kernel (0): identical psi and iteration counts, for both
    directions (two stored graphs) and after an option change (a new
    capture); both match the oracle."""
    import torch

    L, n, rank = 32, 4, 8
    N = L * n
    ph = solver2d.cell_phases_2d_vec(L, 9)
    c = sq.sq2d_build_coeffs(L, n, 9, 0.5, 0.4, 1.0)
    sq.sq2d_coeffs_set_subcell(c, 2)
    V = solver2d.voxel_field_2d(ph, n, 0.4, 1.0, 2)
    psis_o = solver2d.solve_2d(V, tol=1e-13)[0]
    pc = sq.sq2d_precond_setup(N, rank)
    w = sq.sq2d_workspace_create(N)
    outs = {}
    try:
        for mode in (0, 1):
            sq.sq_set_option(sq.SQ_OPT_PCG_GRAPHS, mode)
            runs = []
            for k in range(3):
                if k == 2:
                    sq.sq_set_option(sq.SQ_OPT_MULTIPLIER_TABLE, 1)
                psi = torch.full((N * N,), float(k), dtype=torch.float64, device="cuda")
                info = sq.sq2d_pcg_solve(c, pc, w, k % 2, 1e-12, 4000, psi)
                runs.append((psi.cpu().numpy(), info["iters"], info["status"]))
            outs[mode] = runs
    finally:
        sq.sq_set_option(sq.SQ_OPT_PCG_GRAPHS, 1)
    for k, ((x0, it0, st0), (x1, it1, st1)) in enumerate(zip(outs[0], outs[1])):
        assert st0 == st1 == sq.SQ_OK and it0 == it1
        assert np.array_equal(x0, x1)
        ref = psis_o[k % 2].ravel()
        assert np.linalg.norm(x1 - ref) / np.linalg.norm(ref) <= 1e-9
