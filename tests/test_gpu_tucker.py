"""Canonical preconditioners from given factors and by the paper's Tucker
route (Sec. 4.2), through the C ABI against the oracle: the per-axis factor
tables of pass C (random even nonsymmetric factors), the 2R + 1 split of
Lemma 4.2, HOSVD + Tucker-to-canonical (rank, error, apply at N up to 256),
solves, and argument checks."""
import numpy as np
import pytest

from oracle import pcg, precond, problem, tucker
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


def _even_factors(R, N, seed):
    """Seeded random factors with even rows, f(k) = f(N - k), positive."""
    rng = np.random.default_rng(seed)
    F = rng.uniform(0.2, 1.0, size=(R, N // 2 + 1))
    k = np.arange(N)
    return F[:, np.minimum(k, N - k)]


def _apply(sq, pc, N, r, dt):
    import torch

    prec = sq.SQ_FP64 if dt == "float64" else sq.SQ_FP32_REFINE
    w = sq.sq_workspace_create(N, prec)
    z = torch.empty(N ** 3, dtype=getattr(torch, dt), device="cuda")
    (sq.sq_apply_precond if dt == "float64" else sq.sq_apply_precond_f32)(pc, w, _dev(r.ravel(), dt), z)
    return z.cpu().numpy().astype(np.float64).reshape(N, N, N)


def _relmax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("N", [16, 24, 32, 48, 64, 96, 128])
@pytest.mark.parametrize("R", [3, 8, 13])
def test_nonsymmetric_factors_per_axis(sq, N, R):
    # distinct factors per axis pin which table serves which grid axis
    F = [_even_factors(R, N, 100 * a + R + N) for a in range(3)]
    pc = sq.sq_precond_setup_canonical(N, *F)
    assert sq.sq_precond_info(pc)[0] == R
    G = tucker.canonical_full(*F)
    G[0, 0, 0] = 0.0
    r = inputs.random_field(N, 7 + N)
    ref = precond.apply_precond(G, r)
    assert _relmax(_apply(sq, pc, N, r, "float64"), ref) <= 1e-12
    assert _relmax(_apply(sq, pc, N, r.astype(np.float32), "float32"), ref) <= 3e-5


def test_symmetric_shorthand(sq):
    N, R = 32, 5
    F = _even_factors(R, N, 3)
    a = sq.sq_precond_setup_canonical(N, F)
    b = sq.sq_precond_setup_canonical(N, F, F, F)
    r = inputs.random_field(N, 1)
    assert np.array_equal(_apply(sq, a, N, r, "float64"), _apply(sq, b, N, r, "float64"))


@pytest.mark.parametrize("N,R", [(32, 8), (64, 6), (48, 10)])
def test_lemma_split_equals_projected_exponential_sum(sq, N, R):
    """The 2R + 1 factors of Lemma 4.2 apply the same operator as the R-term
    exponential sum with the zero mode projected out."""
    t, w = precond.rank_r_nodes(N, R)
    pc = sq.sq_precond_setup_canonical(N, *tucker.lemma_split(N, t, w))
    assert sq.sq_precond_info(pc)[0] == 2 * R + 1
    r = inputs.random_field(N, 5)
    ref = precond.apply_precond(precond.core_tensor_from_nodes(N, t, w), r)
    assert _relmax(_apply(sq, pc, N, r, "float64"), ref) <= 1e-12


@pytest.mark.parametrize("N,r,tol", [(24, 5, 0.0), (32, 6, 0.0), (32, 8, 1e-4), (64, 8, 0.0), (96, 10, 1e-3)])
def test_tucker_route_against_oracle(sq, N, r, tol):
    G = precond.core_tensor_exact(N)
    U, _ = tucker.hosvd(G, r)
    F = tucker.tucker_to_canonical(U, tucker.tucker_core(G, U), tol)
    Go = tucker.canonical_full(*F)
    Go[0, 0, 0] = 0.0
    pc = sq.sq_precond_setup_tucker(N, r, tol)
    R, err = sq.sq_precond_info(pc)
    assert R == F[0].shape[0]
    assert abs(err - tucker.max_relative_error_full(N, Go)) <= 1e-9 + 1e-7 * err
    x = inputs.random_field(N, 11)
    ref = precond.apply_precond(Go, x)
    assert _relmax(_apply(sq, pc, N, x, "float64"), ref) <= 1e-9
    assert _relmax(_apply(sq, pc, N, x.astype(np.float32), "float32"), ref) <= 3e-5


def test_tucker_full_size_apply(sq):
    """N = 256, r = 10 (100 terms): the oracle's own HOSVD route, applied
    with its FFT, against the library's factors through pass C."""
    N, r = 256, 10
    G = precond.core_tensor_exact(N)
    U, _ = tucker.hosvd(G, r)
    Go = tucker.canonical_full(*tucker.tucker_to_canonical(U, tucker.tucker_core(G, U), 0.0))
    Go[0, 0, 0] = 0.0
    del G
    pc = sq.sq_precond_setup_tucker(N, r, 0.0)
    x = inputs.random_field(N, 21)
    ref = precond.apply_precond(Go, x)
    assert _relmax(_apply(sq, pc, N, x, "float64"), ref) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solves_with_tucker_preconditioner(sq, prec):
    import torch

    L, n, seed = 4, 8, 17
    N = L * n
    re = problem.realization(L, n, seed, 1.0, 100.0)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
    pc = sq.sq_precond_setup_tucker(N, 8, 1e-4)
    p = sq.SQ_FP64 if prec == "fp64" else sq.SQ_FP32_REFINE
    w = sq.sq_workspace_create(N, p)
    for i in range(3):
        psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
        info = sq.sq_pcg_solve(c, pc, w, i, 1e-11, 3000, p, None, psi)
        assert info["status"] == sq.SQ_OK
        ref = pcg.tight_solve(re.A, re.b[i], N)[0]
        assert np.linalg.norm(psi.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-8


def test_invalid_arguments(sq):
    N = 32
    F = _even_factors(4, N, 9)
    bad = F.copy()
    bad[1, 3] += 0.5  # not even
    with pytest.raises(sq.SqError):
        sq.sq_precond_setup_canonical(N, bad)
    with pytest.raises(sq.SqError):
        sq.sq_precond_setup_canonical(N, F, F, bad)
    with pytest.raises(sq.SqError):
        sq.sq_precond_setup_canonical(N, np.ones((257, N)))  # rank above 256
    for r, tol in ((0, 0.0), (18, 0.0), (8, -1.0), (8, 1.0)):
        with pytest.raises(sq.SqError):
            sq.sq_precond_setup_tucker(N, r, tol)
    with pytest.raises(sq.SqError):
        sq.sq_precond_setup_tucker(48, 17, 0.0)  # 289 terms
    # a Tucker preconditioner has no exponential-sum nodes
    with pytest.raises(sq.SqError):
        sq.sq_precond_factors(sq.sq_precond_setup_tucker(N, 4), 16)


@pytest.mark.parametrize("N,R", [(32, 0), (64, 4), (256, 8), (96, 16)])
def test_info_of_exponential_sums(sq, N, R):
    """sq_precond_info on the default preconditioners: rank, and the relative
    error of the oracle's own exponential sum of that rank."""
    pc = sq.sq_precond_setup(N, R)
    rank, err = sq.sq_precond_info(pc)
    assert rank == R
    if R == 0:
        assert err <= 1e-12
    else:
        assert abs(err - precond.max_relative_error(N, *precond.lsq_nodes(N, R))) <= 1e-9 + 1e-7 * err
