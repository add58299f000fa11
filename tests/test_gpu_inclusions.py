"""Sub-cell inclusions (Sec. 3.1: a centred cube of side sub = 2 alpha n per
cell carries the random value, the rest is a_lo) through the C ABI against
the oracle: RHS, operator (every operator kernel), solves, A_hom, batches."""
import numpy as np
import pytest

from oracle import homogenized, pcg, problem
from tests import inputs

pytestmark = pytest.mark.gpu


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


def _coeffs(sq, L, n, seed, sub, lo=1.0, hi=100.0, p_hi=0.5):
    c = sq.sq_build_coeffs(L, n, seed, p_hi, lo, hi)
    sq.sq_coeffs_set_subcell(c, sub)
    return c


GRIDS = [(4, 4, 2, 1), (3, 8, 4, 2), (4, 8, 2, 3), (6, 8, 6, 4), (12, 4, 2, 5)]


@pytest.mark.parametrize("L,n,sub,seed", GRIDS)
def test_rhs_and_operator_fp64(sq, L, n, sub, seed):
    import torch

    re = problem.realization(L, n, seed, 1.0, 100.0, sub=sub)
    c = _coeffs(sq, L, n, seed, sub)
    N = L * n
    b = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    for i in range(3):
        sq.sq_rhs(c, i, b)
        torch.cuda.synchronize()
        assert np.abs(b.cpu().numpy() - re.b[i]).max() <= 1e-15 * np.abs(re.b[i]).max()
    psi = inputs.random_field(N, seed + 3)
    y = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    sq.sq_apply_operator(c, _dev(psi.ravel()), y)
    torch.cuda.synchronize()
    ref = re.A @ psi.ravel()
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("rows", [1, 4, 8])
@pytest.mark.parametrize("L,n,sub,seed", GRIDS)
def test_operator_fp32_every_kernel(sq, rows, L, n, sub, seed):
    import torch

    re = problem.realization(L, n, seed, 1.0, 100.0, sub=sub)
    c = _coeffs(sq, L, n, seed, sub)
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


@pytest.mark.parametrize("L,n,sub,seed", [(4, 4, 2, 7), (4, 8, 4, 8)])
def test_solves_and_ahom(sq, L, n, sub, seed):
    import torch

    re = problem.realization(L, n, seed, 1.0, 100.0, sub=sub)
    c = _coeffs(sq, L, n, seed, sub)
    N = L * n
    refs = [pcg.tight_solve(re.A, re.b[i], N)[0] for i in range(3)]
    for prec, tol, ptol in ((sq.SQ_FP64, 1e-12, 1e-9), (sq.SQ_FP32_REFINE, 1e-10, 1e-6)):
        pc = sq.sq_precond_setup(N, 0)
        w = sq.sq_workspace_create(N, prec)
        psis = []
        for i in range(3):
            psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
            info = sq.sq_pcg_solve(c, pc, w, i, tol, 4000, prec, None, psi)
            assert info["status"] == sq.SQ_OK
            x = psi.cpu().numpy()
            assert np.linalg.norm(x - refs[i]) / np.linalg.norm(refs[i]) <= ptol
            psis.append(psi)
        Ah, _ = sq.sq_homogenized_matrix(c, *psis)
        Ao = homogenized.ahom_edge(re.a_edges, [r.reshape(N, N, N) for r in refs])
        assert np.abs(Ah - Ao).max() <= 10 * ptol * np.abs(Ao).max()


def test_periodic_array_of_cubes_is_isotropic(sq):
    """Every cell high, alpha = 1/4: a cubic lattice of cubes; by its cubic
    symmetry A_hom = a I exactly (closed form of the structure, any N)."""
    import torch

    L, n, sub = 8, 8, 4
    N = L * n
    c = _coeffs(sq, L, n, 0, sub, lo=0.4, hi=1.0, p_hi=1.0)
    pc = sq.sq_precond_setup(N, 0)
    w = sq.sq_workspace_create(N, sq.SQ_FP64)
    psis = [torch.empty(N ** 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    for i in range(3):
        assert sq.sq_pcg_solve(c, pc, w, i, 1e-12, 4000, sq.SQ_FP64, None, psis[i])["status"] == sq.SQ_OK
    A, E = sq.sq_homogenized_matrix(c, *psis)
    assert np.abs(A - np.diag(np.diag(A))).max() <= 1e-10
    assert np.abs(np.diag(A) - A[0, 0]).max() <= 1e-10
    assert 0.4 < A[0, 0] < 0.4 + 0.6 / 8  # between a_lo and the arithmetic mean (inclusion volume 1/8)


def test_batch_with_inclusions(sq):
    import torch

    descs, pl, singles = [], [], []
    for L, n, sub, seed in [(8, 4, 2, 31), (12, 4, 2, 32), (4, 8, 4, 33)]:
        N = L * n
        c = _coeffs(sq, L, n, seed, sub, lo=1.0, hi=10.0)
        pc = sq.sq_precond_setup(N, 0)
        w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
        ps = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
        sq.sq_pcg_solve(c, pc, w, 0, 1e-9, 3000, sq.SQ_FP32_REFINE, None, ps)
        singles.append(ps.cpu().numpy())
        descs.append((c, 0, torch.empty(N ** 3, dtype=torch.float64, device="cuda")))
        pl.append(pc)
    infos = sq.sq_pcg_solve_batched(sq.sq_batch_create(descs, pl), 1e-9, 3000)
    for (c, i, psi), xs, inf in zip(descs, singles, infos):
        assert inf["status"] == sq.SQ_OK
        x = psi.cpu().numpy()
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-6


def test_invalid_subcell(sq):
    c = sq.sq_build_coeffs(4, 8, 1, 0.5, 1.0, 10.0)
    for sub in (0, 9, 3):
        with pytest.raises(sq.SqError):
            sq.sq_coeffs_set_subcell(c, sub)
    sq.sq_coeffs_set_subcell(c, 8)  # the whole cell is allowed
