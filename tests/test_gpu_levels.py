"""Multi-level media (varying contrast, Sec. 2: inclusion cells carry
lambda + beta_c with a contrast that differs between cells) through the C ABI
against the oracle: level draw, RHS, every operator kernel, solves, A_hom,
batches, the laminate closed form and sampled nodes at N = 256."""
import numpy as np
import pytest

from oracle import assembly, homogenized, pcg, problem, rng
from tests import inputs

pytestmark = pytest.mark.gpu

VALS3 = (0.4, 0.7, 1.0)  # lambda = 0.4, contrasts beta = 0.3 and 0.6
PROBS3 = (0.5, 0.25, 0.25)
VALS4 = (1.0, 30.0, 4.0, 100.0)
PROBS4 = (0.4, 0.2, 0.3, 0.1)


@pytest.fixture(scope="module")
def sq():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2007_06524_gb300 as pkg

    return pkg


def _dev(a, dtype="float64"):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=getattr(torch, dtype))


def _coeffs(sq, L, n, seed, probs, vals, sub=None):
    c = sq.sq_build_coeffs_levels(L, n, seed, probs, vals)
    if sub is not None:
        sq.sq_coeffs_set_subcell(c, sub)
    return c


def _oracle(L, n, seed, probs, vals, sub=None):
    return problem.realization_levels(L, n, seed, vals, probs=probs, sub=sub)


@pytest.mark.parametrize("probs", [PROBS3, PROBS4, (0.0, 0.5, 0.5), (0.25, 0.75)])
@pytest.mark.parametrize("L,seed", [(6, 1), (24, 2), (64, 2**63 + 9)])
def test_level_draw_bit_exact(sq, probs, L, seed):
    c = sq.sq_build_coeffs_levels(L, 2, seed, probs, (1.0,) * len(probs))
    got, n_hi = sq.sq_coeffs_cells(c)
    want = rng.cell_levels(L, seed, probs) if L <= 6 else rng.cell_levels_vec(L, seed, probs)
    assert np.array_equal(got, want) and n_hi == int((want > 0).sum())
    # redraw in place with another seed
    sq.sq_coeffs_regenerate_levels(c, seed + 1, probs)
    got, _ = sq.sq_coeffs_cells(c)
    assert np.array_equal(got, rng.cell_levels_vec(L, seed + 1, probs))


def test_two_levels_match_the_checkerboard_handle(sq):
    import torch

    a = sq.sq_build_coeffs(8, 4, 77, 0.3, 1.0, 10.0)
    b = sq.sq_build_coeffs_levels(8, 4, 77, (0.7, 0.3), (1.0, 10.0))
    assert np.array_equal(sq.sq_coeffs_cells(a)[0], sq.sq_coeffs_cells(b)[0])
    x = _dev(inputs.random_field(32, 4).ravel())
    ya, yb = torch.empty_like(x), torch.empty_like(x)
    sq.sq_apply_operator(a, x, ya)
    sq.sq_apply_operator(b, x, yb)
    assert torch.equal(ya, yb)


GRIDS = [(4, 4, None, 1), (3, 8, 4, 2), (4, 8, None, 3), (6, 8, 6, 4), (12, 4, 2, 5), (2, 16, 8, 6)]


@pytest.mark.parametrize("K", [3, 4])
@pytest.mark.parametrize("L,n,sub,seed", GRIDS)
def test_rhs_and_operator_fp64(sq, K, L, n, sub, seed):
    import torch

    probs, vals = (PROBS3, VALS3) if K == 3 else (PROBS4, VALS4)
    re = _oracle(L, n, seed, probs, vals, sub)
    c = _coeffs(sq, L, n, seed, probs, vals, sub)
    N = L * n
    b = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    for i in range(3):
        sq.sq_rhs(c, i, b)
        torch.cuda.synchronize()
        assert np.abs(b.cpu().numpy() - re.b[i]).max() <= 4e-15 * max(vals)
    psi = inputs.random_field(N, seed + 3)
    y = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    sq.sq_apply_operator(c, _dev(psi.ravel()), y)
    torch.cuda.synchronize()
    ref = re.A @ psi.ravel()
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("rows", [1, 2, 4, 8])
@pytest.mark.parametrize("L,n,sub,seed", GRIDS)
def test_operator_fp32_every_kernel(sq, rows, L, n, sub, seed):
    import torch

    re = _oracle(L, n, seed, PROBS4, VALS4, sub)
    c = _coeffs(sq, L, n, seed, PROBS4, VALS4, sub)
    N = L * n
    psi = inputs.random_field(N, seed + 5, np.float32)
    y = torch.empty(N ** 3, dtype=torch.float32, device="cuda")
    try:
        sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, rows)
        sq.sq_apply_operator_f32(c, _dev(psi.ravel(), "float32"), y)
        torch.cuda.synchronize()
    finally:
        sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, 0)
    ref = re.A @ psi.ravel().astype(np.float64)
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_host_levels_and_relabelling(sq):
    """Host levels (a byte past the top level reads as the top level), then
    new values for the same handle through set_levels: the oracle's field
    each time."""
    import torch

    L, n = 4, 8
    lv = rng.cell_levels(L, 12, (0.3, 0.3, 0.4))
    raw = lv.copy()
    raw[raw == 2] = 200
    c = sq.sq_coeffs_from_host_levels(L, n, raw.ravel(), (5.0, 1.0, 2.0))
    got, _ = sq.sq_coeffs_cells(c)
    assert np.array_equal(got, lv)
    sq.sq_coeffs_set_subcell(c, 4)
    psi = inputs.random_field(L * n, 6)
    y = torch.empty(psi.size, dtype=torch.float64, device="cuda")
    for vals in ((5.0, 1.0, 2.0), VALS3):
        sq.sq_coeffs_set_levels(c, vals)
        re = problem.realization_levels(L, n, 0, vals, level=lv, sub=4)
        sq.sq_apply_operator(c, _dev(psi.ravel()), y)
        ref = re.A @ psi.ravel()
        assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("L,n,sub,seed", [(4, 4, None, 7), (4, 8, 4, 8), (3, 8, 2, 9)])
def test_solves_and_ahom(sq, L, n, sub, seed):
    import torch

    re = _oracle(L, n, seed, PROBS3, VALS3, sub)
    c = _coeffs(sq, L, n, seed, PROBS3, VALS3, sub)
    N = L * n
    refs = [pcg.tight_solve(re.A, re.b[i], N)[0] for i in range(3)]
    Ao = homogenized.ahom_edge(re.a_edges, [r.reshape(N, N, N) for r in refs])
    for prec, rank, tol, ptol in ((sq.SQ_FP64, 0, 1e-12, 1e-9), (sq.SQ_FP64, 8, 1e-12, 1e-9),
                                  (sq.SQ_FP32_REFINE, 0, 1e-10, 1e-6), (sq.SQ_FP32_REFINE, 8, 1e-10, 1e-6)):
        pc = sq.sq_precond_setup(N, rank)
        w = sq.sq_workspace_create(N, prec)
        psis = []
        for i in range(3):
            psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
            info = sq.sq_pcg_solve(c, pc, w, i, tol, 4000, prec, None, psi)
            assert info["status"] == sq.SQ_OK
            x = psi.cpu().numpy()
            assert np.linalg.norm(x - refs[i]) / np.linalg.norm(refs[i]) <= ptol
            psis.append(psi)
        Ah, Ae = sq.sq_homogenized_matrix(c, *psis)
        assert np.abs(Ah - Ao).max() <= 10 * ptol * np.abs(Ao).max()
        assert np.abs(Ae - Ao).max() <= 10 * ptol * np.abs(Ao).max()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_layer_type_laminate_closed_form(sq, axis):
    """Layer-type medium with two contrasts (levels set per layer of cells
    along one axis): A_hom = diag(harmonic / arithmetic means), exactly."""
    import torch

    L, n = 16, 4
    N = L * n
    layer = np.array([1, 2] * (L // 2), dtype=np.uint8)
    layer[[3, 7, 12]] = 0  # three background layers
    shape = [1, 1, 1]
    shape[axis] = L
    lv = np.broadcast_to(layer.reshape(shape), (L, L, L)).copy()
    c = sq.sq_coeffs_from_host_levels(L, n, lv.ravel(), VALS3)
    pc = sq.sq_precond_setup(N, 0)
    w = sq.sq_workspace_create(N, sq.SQ_FP64)
    psis = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    for i in range(3):
        assert sq.sq_pcg_solve(c, pc, w, i, 1e-13, 4000, sq.SQ_FP64, None, psis[i])["status"] == sq.SQ_OK
    A, E = sq.sq_homogenized_matrix(c, *psis)
    v = np.array(VALS3)[layer]
    want = np.full(3, v.mean())
    want[axis] = 1.0 / np.mean(1.0 / v)
    assert np.abs(np.diag(A) - want).max() <= 1e-11
    assert np.abs(A - np.diag(np.diag(A))).max() <= 1e-11
    assert np.abs(E - A).max() <= 1e-10


def test_batch_mixed_levels_against_oracle(sq):
    """A batch mixing two-, three- and four-level media (tables sized for the
    largest) reproduces the oracle's solutions."""
    import torch

    cases = [(8, 4, None, 31, (0.5, 0.5), (1.0, 10.0)), (12, 4, 2, 32, PROBS3, VALS3),
             (4, 8, 4, 33, PROBS4, VALS4), (2, 16, None, 34, PROBS3, VALS3)]
    descs, pl, refs = [], [], []
    for L, n, sub, seed, probs, vals in cases:
        N = L * n
        c = _coeffs(sq, L, n, seed, probs, vals, sub)
        re = _oracle(L, n, seed, probs, vals, sub)
        refs.append(pcg.tight_solve(re.A, re.b[1], N)[0])
        descs.append((c, 1, torch.empty(N ** 3, dtype=torch.float64, device="cuda")))
        pl.append(sq.sq_precond_setup(N, 0))
    infos = sq.sq_pcg_solve_batched(sq.sq_batch_create(descs, pl), 1e-10, 3000)
    for (c, i, psi), xr, inf in zip(descs, refs, infos):
        assert inf["status"] == sq.SQ_OK
        x = psi.cpu().numpy()
        assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6


def test_full_size_sampled_nodes(sq):
    """N = 256 (L = 32, n = 8), two contrasts on whole cells: operator, RHS and
    residual at sampled nodes against the oracle's one-node formulas."""
    import torch

    L, n = 32, 8
    N = L * n
    c = _coeffs(sq, L, n, 2024, PROBS3, VALS3)
    cellval = rng.level_values(rng.cell_levels_vec(L, 2024, PROBS3), VALS3)
    psi = inputs.random_field(N, 99)
    y = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    sq.sq_apply_operator(c, _dev(psi.ravel()), y)
    b = torch.empty_like(y)
    sq.sq_rhs(c, 2, b)
    yh, bh = y.cpu().numpy().reshape(N, N, N), b.cpu().numpy().reshape(N, N, N)
    for j in inputs.sample_nodes(N, 48, 5):
        ref = assembly.apply_at(cellval, n, lambda k: psi[k], j)
        assert abs(yh[j] - ref) <= 1e-12 * max(1.0, abs(ref))
        assert abs(bh[j] - assembly.rhs_at(cellval, n, 2, j)) <= 4e-15


def test_full_size_solve_properties(sq):
    """N = 256 with alpha = 1/4 inclusions and two contrasts (no oracle solve
    at this size): the recomputed FP64 residual meets the tolerance, A_hom is
    symmetric, its edge and energy forms agree, and each diagonal entry lies
    between the harmonic and arithmetic means of its edge coefficients."""
    import torch

    L, n, sub = 32, 8, 4
    N = L * n
    c = _coeffs(sq, L, n, 11, PROBS3, VALS3, sub)
    pc = sq.sq_precond_setup(N, 8)
    w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
    psis = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    for i in range(3):
        info = sq.sq_pcg_solve(c, pc, w, i, 1e-8, 2000, sq.SQ_FP32_REFINE, None, psis[i])
        assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-8
    A, E = sq.sq_homogenized_matrix(c, *psis)
    assert np.abs(A - A.T).max() <= 1e-6 and np.abs(A - E).max() <= 1e-6
    lv = rng.cell_levels_vec(L, 11, PROBS3)
    V = assembly.level_field(lv, n, VALS3, sub)
    a_edges = assembly.edge_coefficients_voxels(V)
    for i in range(3):
        lo = 1.0 / np.mean(1.0 / a_edges[i])
        hi = a_edges[i].mean()
        assert lo - 1e-9 <= A[i, i] <= hi + 1e-9


def test_invalid_levels(sq):
    c = sq.sq_build_coeffs(4, 8, 1, 0.5, 1.0, 10.0)
    for vals in ((1.0, 0.0, 2.0), (1.0, -1.0), (1.0, float("inf"), 2.0)):
        with pytest.raises(sq.SqError):
            sq.sq_coeffs_set_levels(c, vals)
    with pytest.raises(ValueError):
        sq.sq_coeffs_set_levels(c, (1.0,) * 5)
    with pytest.raises(sq.SqError):
        sq.sq_build_coeffs_levels(4, 8, 1, (0.5, 0.2, 0.2), VALS3)  # probabilities sum to 0.9
    with pytest.raises(sq.SqError):
        sq.sq_build_coeffs_levels(4, 8, 1, (0.5, 0.6, -0.1), VALS3)
    d = sq.sq_build_coeffs_levels(4, 8, 1, PROBS3, VALS3)
    with pytest.raises(sq.SqError):
        sq.sq_coeffs_regenerate_levels(d, 2, PROBS4)  # level count differs from the handle's
