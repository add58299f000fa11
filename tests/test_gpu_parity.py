"""GPU parity: libsq (through its C ABI) against the CPU oracle.

Tolerances: bit-exact for the cell phases; FP64 operator / RHS / preconditioner
within a few ulps of the field scale (1e-13 relative); FP64 solves run to
rel. residual 1e-12 so the solution matches the oracle's tight solve within
1e-9 (rel. L2) and A_hom within 1e-10; FP32 kernels within 1e-5 relative;
FP32 + FP64 refinement to 1e-10 within 1e-6 of the oracle.
"""
import functools

import numpy as np
import pytest

from oracle import assembly, homogenized, pcg, precond, problem, rng
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


def _host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def _relmax(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# ------------------------------------------------------------------ cells
@pytest.mark.parametrize("L,n,seed,p", [(4, 4, 0, 0.5), (6, 2, 3, 0.5), (6, 2, 11, 0.3), (32, 8, 0, 0.5),
                                        (32, 8, 7, 0.5), (64, 8, 1, 0.5), (4, 2, 2**63 + 9, 0.9)])
def test_cell_phases_bit_exact(sq, L, n, seed, p):
    c = sq.sq_build_coeffs(L, n, seed, p, 1.0, 10.0)
    ph, nhi = sq.sq_coeffs_cells(c)
    ref = rng.cell_phases(L, seed, p) if L <= 6 else rng.cell_phases_vec(L, seed, p)
    assert np.array_equal(ph, ref)
    assert nhi == int(ref.sum())


def test_cells_from_host_roundtrip(sq):
    ph = rng.cell_phases_vec(8, 5)
    c = sq.sq_coeffs_from_host(8, 4, ph * 7, 1.0, 100.0)  # nonzero = high
    out, nhi = sq.sq_coeffs_cells(c)
    assert np.array_equal(out, ph) and nhi == int(ph.sum())


# --------------------------------------------------------- operator, RHS
GRIDS = [(4, 4, 0), (3, 4, 1), (4, 8, 2), (12, 4, 3), (6, 8, 4), (24, 4, 5), (2, 6, 6)]


@pytest.mark.parametrize("L,n,seed", GRIDS)
def test_rhs_and_operator_fp64(sq, L, n, seed):
    re = problem.realization(L, n, seed, 1.0, 100.0)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
    N = L * n
    import torch

    b = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    for i in range(3):
        sq.sq_rhs(c, i, b)
        assert _relmax(_host(b), re.b[i]) <= 1e-15
    psi = inputs.random_field(N, seed + 100)
    y = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    sq.sq_apply_operator(c, _dev(psi.ravel()), y)
    assert _relmax(_host(y), re.A @ psi.ravel()) <= 1e-13


@pytest.mark.parametrize("L,n,seed", GRIDS[:4])
def test_operator_fp32(sq, L, n, seed):
    re = problem.realization(L, n, seed, 1.0, 100.0)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
    N = L * n
    import torch

    psi = inputs.random_field(N, seed + 7, np.float32)
    y = torch.empty(N ** 3, dtype=torch.float32, device="cuda")
    sq.sq_apply_operator_f32(c, _dev(psi.ravel(), "float32"), y)
    assert _relmax(_host(y).astype(np.float64), re.A @ psi.ravel().astype(np.float64)) <= 1e-5


# FP32 operator with 1, 2 and 4 node rows per thread and the shared-memory-
# staged kernel (8; used where N is a multiple of 32, else 4 rows): grids
# ragged against the 32-wide j3 tiles and the 8*rows-high j2 tiles, and exact
# multiples (every valid N, 2^a 3^b with b <= 1 and N >= 8, is divisible by 4).
ROW_GRIDS = [(3, 4, 8), (3, 8, 9), (4, 8, 11), (12, 4, 12), (12, 8, 13), (6, 32, 14), (16, 2, 15), (8, 4, 16),
             (4, 16, 17)]


@pytest.mark.parametrize("rows", [1, 2, 4, 8])
@pytest.mark.parametrize("L,n,seed", ROW_GRIDS)
def test_operator_fp32_rows_per_thread(sq, rows, L, n, seed):
    re = problem.realization(L, n, seed, 1.0, 100.0)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
    N = L * n
    import torch

    psi = inputs.random_field(N, seed + 17, np.float32)
    y = torch.empty(N ** 3, dtype=torch.float32, device="cuda")
    try:
        sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, rows)
        sq.sq_apply_operator_f32(c, _dev(psi.ravel(), "float32"), y)
    finally:
        sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, 0)
    assert _relmax(_host(y).astype(np.float64), re.A @ psi.ravel().astype(np.float64)) <= 1e-5


@pytest.mark.parametrize("zc", [4, 7, 64])
def test_staged_operator_plane_runs(sq, zc):
    """The staged FP32 operator with a tuned plane run per block (4, 7 which
    does not divide N, and the whole axis) against the oracle's operator."""
    import torch

    L, n, seed = 8, 8, 5
    N = L * n
    re = problem.realization(L, n, seed, 1.0, 100.0)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
    psi = inputs.random_field(N, seed + 3, np.float32)
    y = torch.empty(N ** 3, dtype=torch.float32, device="cuda")
    try:
        sq.sq_set_tiles([(N, 0, zc, 8)])
        sq.sq_apply_operator_f32(c, _dev(psi.ravel(), "float32"), y)
    finally:
        sq.sq_set_tiles([])
    assert _relmax(_host(y).astype(np.float64), re.A @ psi.ravel().astype(np.float64)) <= 1e-5


@pytest.mark.parametrize("rows", [1, 2, 4, 8])
def test_fp32_refinement_rows_per_thread(sq, rows):
    # p.Ap of the inner FP32 iteration comes from the operator's reduction
    re = problem.realization(6, 4, 21, 1.0, 100.0)
    c = sq.sq_build_coeffs(6, 4, 21, 0.5, 1.0, 100.0)
    ref = pcg.tight_solve(re.A, re.b[0], re.N)[0]
    try:
        sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, rows)
        psi, info = _solve(sq, c, re.N, 0, 0, 1e-10, precision=sq.SQ_FP32_REFINE)
    finally:
        sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, 0)
    assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-10
    x = _host(psi)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-6


def test_stencil_rows_option_rejects_bad_values(sq):
    for bad in (3, 5, -1, 16):
        with pytest.raises(sq.SqError):
            sq.sq_set_option(sq.SQ_OPT_STENCIL_ROWS, bad)


# ---------------------------------------------------------- preconditioner
# The oracle's own exponential sum (geometric nodes, numpy least-squares
# weights): the expected G of every rank-R test comes from here, never from
# the library's factors.
_oracle_nodes = functools.lru_cache(maxsize=None)(precond.lsq_nodes)


def _core(sq, pc, N, rank):
    """The oracle's G for a preconditioner of the given rank: the exact
    Fourier diagonal, or the oracle's rank-R exponential sum."""
    if rank == 0:
        return precond.core_tensor_exact(N)
    return precond.core_tensor_from_nodes(N, *_oracle_nodes(N, rank))


@pytest.mark.parametrize("N,rank", [(8, 4), (16, 6), (32, 8), (64, 16), (256, 8), (256, 4), (256, 16), (48, 4),
                                    (96, 8), (512, 8), (64, 32), (16, 40), (16, 16), (24, 32), (12, 16)])
def test_rank_r_factors_match_oracle_construction(sq, N, rank):
    """The library's nodes and weights against the oracle's independent
    construction: same geometric nodes, and an exponential sum that agrees
    on every distinct eigenvalue of the Laplacian to 1e-12 (the weights
    themselves only to the conditioning of the least-squares problem)."""
    pc = sq.sq_precond_setup(N, rank)
    t, w = sq.sq_precond_factors(pc, rank)
    to, wo = _oracle_nodes(N, rank)
    assert np.all(w > 0) and np.all(t > 0)
    assert np.abs(t / to - 1).max() <= 1e-13
    assert np.abs(w / wo - 1).max() <= 1e-8
    x = precond.spectrum_values(N)
    g, go = np.exp(-np.outer(x, t)) @ w, np.exp(-np.outer(x, to)) @ wo
    assert np.abs(g / go - 1).max() <= 1e-12


@pytest.mark.parametrize("N", [8, 12, 16, 24, 32, 48, 64, 96, 128])
@pytest.mark.parametrize("rank", [0, 6, 16])
def test_precond_fp64(sq, N, rank):
    import torch

    pc = sq.sq_precond_setup(N, rank)
    w = sq.sq_workspace_create(N, sq.SQ_FP64)
    r = inputs.random_field(N, N + rank)
    z = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    sq.sq_apply_precond(pc, w, _dev(r.ravel()), z)
    ref = precond.apply_precond(_core(sq, pc, N, rank), r)
    assert _relmax(_host(z).reshape(N, N, N), ref) <= 1e-12


@pytest.mark.parametrize("N", [16, 48, 96, 256])
@pytest.mark.parametrize("rank", [0, 8])
def test_precond_fp32(sq, N, rank):
    import torch

    pc = sq.sq_precond_setup(N, rank)
    w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
    r = inputs.random_field(N, 3 * N + rank, np.float32)
    z = torch.empty(N ** 3, dtype=torch.float32, device="cuda")
    sq.sq_apply_precond_f32(pc, w, _dev(r.ravel(), "float32"), z)
    ref = precond.apply_precond(_core(sq, pc, N, rank), r.astype(np.float64))
    assert _relmax(_host(z).reshape(N, N, N).astype(np.float64), ref) <= 2e-5


def test_precond_fp64_full_size(sq):
    import torch

    N, rank = 256, 8
    pc = sq.sq_precond_setup(N, rank)
    w = sq.sq_workspace_create(N, sq.SQ_FP64)
    r = inputs.random_field(N, 42)
    z = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    sq.sq_apply_precond(pc, w, _dev(r.ravel()), z)
    ref = precond.apply_precond(_core(sq, pc, N, rank), r)
    assert _relmax(_host(z).reshape(N, N, N), ref) <= 1e-12


# ------------------------------------------------------------------ solves
def _solve(sq, c, N, dir, rank, tol, precision=0, max_iter=2000, x0=None):
    import torch

    pc = sq.sq_precond_setup(N, rank)
    w = sq.sq_workspace_create(N, precision)
    psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    info = sq.sq_pcg_solve(c, pc, w, dir, tol, max_iter, precision, x0, psi)
    return psi, info


@pytest.mark.parametrize("rank", [0, 6])
def test_solve_plain_n16(sq, rank):
    # L=4, n=4, Bernoulli(1/2) on {1,10}, seed 0, e_1
    re = problem.realization(4, 4, 0, 1.0, 10.0)
    ref, it_tight, _ = pcg.tight_solve(re.A, re.b[0], re.N)
    c = sq.sq_build_coeffs(4, 4, 0, 0.5, 1.0, 10.0)
    psi, info = _solve(sq, c, re.N, 0, rank, 1e-12)
    x = _host(psi)
    assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-12
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-9
    assert abs(x.mean()) < 1e-14
    # iteration count of the same PCG on the oracle at tol 1e-10
    G = _core(sq, sq.sq_precond_setup(re.N, rank), re.N, rank)
    P = lambda r: precond.apply_precond(G, r.reshape(re.N, re.N, re.N)).ravel()  # noqa: E731
    _, it_o, _ = pcg.pcg(re.A, re.b[0], P, tol=1e-10)
    psi2, info2 = _solve(sq, c, re.N, 0, rank, 1e-10)
    assert abs(info2["iters"] - it_o) <= 1
    Ah, _ = sq.sq_homogenized_matrix(c, psi, psi, psi)
    Ao = homogenized.ahom_edge(re.a_edges, [ref.reshape(re.N, re.N, re.N), None, None])
    assert abs(Ah[0, 0] - Ao[0, 0]) <= 1e-10 * abs(Ao[0, 0])


@pytest.mark.parametrize("L,n,seed,rank", [(4, 4, 1, 8), (12, 4, 2, 0), (6, 8, 3, 4)])
def test_solve_three_dirs_ahom(sq, L, n, seed, rank):
    re = problem.realization(L, n, seed, 1.0, 100.0)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
    N = re.N
    psis, refs = [], []
    for i in range(3):
        ref = pcg.tight_solve(re.A, re.b[i], N)[0]
        psi, info = _solve(sq, c, N, i, rank, 1e-12)
        assert info["status"] == sq.SQ_OK
        x = _host(psi)
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-9
        psis.append(psi)
        refs.append(ref.reshape(N, N, N))
    Ah, Ae = sq.sq_homogenized_matrix(c, *psis)
    Ao = homogenized.ahom_edge(re.a_edges, refs)
    Aeo = homogenized.ahom_energy(re.a_edges, refs)
    assert np.abs(Ah - Ao).max() <= 1e-10 * np.abs(Ao).max()
    assert np.abs(Ae - Aeo).max() <= 1e-10 * np.abs(Ao).max()
    assert np.abs(Ah - Ah.T).max() <= 1e-10 * np.abs(Ah).max()


def test_fp32_refinement(sq):
    re = problem.realization(4, 8, 5, 1.0, 100.0)
    c = sq.sq_build_coeffs(4, 8, 5, 0.5, 1.0, 100.0)
    ref = pcg.tight_solve(re.A, re.b[1], re.N)[0]
    psi, info = _solve(sq, c, re.N, 1, 0, 1e-10, precision=sq.SQ_FP32_REFINE)
    assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-10
    assert info["outer_steps"] >= 2
    x = _host(psi)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-6
    assert abs(x.mean()) <= 1e-12 * np.abs(x).max()


def test_warm_start_and_enoconv(sq):
    re = problem.realization(4, 4, 3, 1.0, 10.0)
    c = sq.sq_build_coeffs(4, 4, 3, 0.5, 1.0, 10.0)
    ref = pcg.tight_solve(re.A, re.b[2], re.N)[0]
    psi, info = _solve(sq, c, re.N, 2, 0, 1e-8, max_iter=2)
    assert info["status"] == sq.SQ_ENOCONV and info["iters"] == 2
    x0 = _dev(ref + 1e-6 * inputs.random_field(re.N, 1).ravel())
    psi, info_w = _solve(sq, c, re.N, 2, 0, 1e-8, x0=x0)
    _, info_0 = _solve(sq, c, re.N, 2, 0, 1e-8)
    assert info_w["used_guess"] == 1 and info_w["iters"] < info_0["iters"]
    assert np.linalg.norm(_host(psi) - ref) / np.linalg.norm(ref) <= 1e-7


def test_degenerate_constant_coefficient(sq):
    c = sq.sq_build_coeffs(4, 4, 0, 0.5, 3.0, 3.0)   # a_lo == a_hi -> b = 0
    psi, info = _solve(sq, c, 16, 0, 0, 1e-8)
    assert info["status"] == sq.SQ_OK and info["iters"] == 0
    assert np.abs(_host(psi)).max() == 0.0
    Ah, _ = sq.sq_homogenized_matrix(c, psi, psi, psi)
    assert np.allclose(Ah, 3.0 * np.eye(3), atol=1e-14)


def test_invalid_arguments(sq):
    with pytest.raises(sq.SqError) as e:
        sq.sq_build_coeffs(5, 2, 0, 0.5, 1.0, 10.0)      # N = 10 not 2^a 3^b
    assert e.value.status == sq.SQ_EINVAL
    with pytest.raises(sq.SqError):
        sq.sq_precond_setup(16, 1)
    with pytest.raises(sq.SqError):
        sq.sq_workspace_create(1024, 0)
    c = sq.sq_build_coeffs(4, 4, 0, 0.5, 1.0, 10.0)
    pc = sq.sq_precond_setup(32, 0)
    w = sq.sq_workspace_create(16, 0)
    import torch

    psi = torch.zeros(16 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SqError):
        sq.sq_pcg_solve(c, pc, w, 0, 1e-8, 10, 0, None, psi)
    with pytest.raises(sq.SqError):
        sq.sq_pcg_solve(c, sq.sq_precond_setup(16, 0), w, 0, 1e-8, 10, sq.SQ_FP32_REFINE, None, psi)


# --------------------------------------- full size (L=32, n=8, N=256), sampled
def test_full_size_n256_sampled(sq):
    import torch

    L, n, seed = 32, 8, 0
    N = L * n
    cellval = rng.cell_values(rng.cell_phases_vec(L, seed), 1.0, 100.0)
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
    nodes = inputs.sample_nodes(N, 300, 1)
    # operator on a random field, sampled
    psi_h = inputs.random_field(N, 9)
    y = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    sq.sq_apply_operator(c, _dev(psi_h.ravel()), y)
    yh = _host(y).reshape(N, N, N)
    for j in nodes:
        ref = assembly.apply_at(cellval, n, lambda k: psi_h[k], j)
        assert abs(yh[j] - ref) <= 1e-13 * (abs(ref) + 100.0)
    # RHS, sampled
    b = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    sq.sq_rhs(c, 1, b)
    bh = _host(b).reshape(N, N, N)
    for j in nodes:
        assert bh[j] == assembly.rhs_at(cellval, n, 1, j)
    # the timed solve: FP64 PCG, rank-8 preconditioner, tol 1e-8, all three directions
    psis = []
    for i in range(3):
        psi, info = _solve(sq, c, N, i, 8, 1e-8)
        assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-8
        assert 10 <= info["iters"] <= 200
        psis.append(psi)
    Ah, Ae = sq.sq_homogenized_matrix(c, *psis)
    vals = cellval.ravel()
    hm, am = 1.0 / np.mean(1.0 / vals), vals.mean()
    for i in range(3):
        assert hm <= Ah[i, i] <= am
    assert np.abs(Ah - Ah.T).max() <= 1e-6 * Ah[0, 0]
    assert np.abs(Ah - Ae).max() <= 1e-6 * Ah[0, 0]
    # the residual of the returned psi_1 checked at sampled nodes by the oracle
    x = _host(psis[0]).reshape(N, N, N)
    for j in nodes[:50]:
        rj = assembly.rhs_at(cellval, n, 0, j) - assembly.apply_at(cellval, n, lambda k: x[k], j)
        assert abs(rj) <= 1e-3  # pointwise residual of a 1e-8 relative solve (||b|| ~ 1e4)
    # FP32 + FP64 refinement on the same system agrees with the FP64 solve
    psi_r, info_r = _solve(sq, c, N, 0, 0, 1e-8, precision=sq.SQ_FP32_REFINE)
    assert info_r["status"] == sq.SQ_OK
    xr = _host(psi_r)
    assert np.linalg.norm(xr - x.ravel()) / np.linalg.norm(x) <= 1e-5


@pytest.mark.parametrize("N", [16, 32, 48, 64, 96, 128, 256])
def test_precond_generic_and_two_stage_paths_agree(sq, N):
    """The Hartley passes have two implementations (two-stage register plans
    for x1/x2 and for the contiguous x3, and the generic shared-memory
    Stockham tile); both must give the oracle's result."""
    import torch

    rank = 8
    pc = sq.sq_precond_setup(N, rank)
    G = _core(sq, pc, N, rank)
    for prec, dt, tol in ((sq.SQ_FP64, "float64", 1e-12), (sq.SQ_FP32_REFINE, "float32", 2e-5)):
        w = sq.sq_workspace_create(N, prec)
        r = inputs.random_field(N, 7 * N, np.float64 if dt == "float64" else np.float32)
        ref = precond.apply_precond(G, r.astype(np.float64))
        outs = []
        for opt in (0, 1, 2):
            sq.sq_set_option(sq.SQ_OPT_STRIDED_TWO_STAGE, opt)
            z = torch.empty(N ** 3, dtype=getattr(torch, dt), device="cuda")
            (sq.sq_apply_precond if dt == "float64" else sq.sq_apply_precond_f32)(pc, w, _dev(r.ravel(), dt), z)
            outs.append(_host(z).reshape(N, N, N).astype(np.float64))
        sq.sq_set_option(sq.SQ_OPT_STRIDED_TWO_STAGE, 1)
        for z in outs:
            assert _relmax(z, ref) <= tol


def test_refinement_n128_against_oracle(sq):
    """The precision configuration's oracle subsample: L=16, n=8 (N=128),
    Bernoulli(1/2) on {1,100}, FP32 PCG inside FP64 refinement to 1e-10: error
    against the FP64 oracle's tight solve <= 1e-6 (stated per result)."""
    re = problem.realization(16, 8, 0, 1.0, 100.0)
    ref = pcg.tight_solve(re.A, re.b[0], re.N)[0]
    c = sq.sq_build_coeffs(16, 8, 0, 0.5, 1.0, 100.0)
    for rank in (0, 8):
        psi, info = _solve(sq, c, re.N, 0, rank, 1e-10, precision=sq.SQ_FP32_REFINE, max_iter=4000)
        assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-10
        err = np.linalg.norm(_host(psi) - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (rank, err)


@pytest.mark.parametrize("opt", [0, 1, 2])
def test_solves_with_each_pass_implementation(sq, opt):
    """The fused PCG forms of the x3 passes (r -= alpha q with ||r||^2 on
    load, x += alpha p and p = z + beta p on store) in both implementations:
    FP32 refinement and FP64 solves reach the oracle's corrector."""
    re = problem.realization(8, 8, 33, 1.0, 100.0)
    c = sq.sq_build_coeffs(8, 8, 33, 0.5, 1.0, 100.0)
    ref = pcg.tight_solve(re.A, re.b[2], re.N)[0]
    try:
        sq.sq_set_option(sq.SQ_OPT_STRIDED_TWO_STAGE, opt)
        psi32, i32 = _solve(sq, c, re.N, 2, 8, 1e-10, precision=sq.SQ_FP32_REFINE)
        psi64, i64 = _solve(sq, c, re.N, 2, 8, 1e-12)
    finally:
        sq.sq_set_option(sq.SQ_OPT_STRIDED_TWO_STAGE, 1)
    assert i32["status"] == sq.SQ_OK and i32["relres_true"] <= 1e-10
    assert i64["status"] == sq.SQ_OK and i64["relres_true"] <= 1e-12
    assert np.linalg.norm(_host(psi32) - ref) / np.linalg.norm(ref) <= 1e-6
    assert np.linalg.norm(_host(psi64) - ref) / np.linalg.norm(ref) <= 1e-9


@pytest.mark.parametrize("N", [256, 512])
@pytest.mark.parametrize("rank", [0, 8])
def test_precond_cosine_modes_full_size(sq, N, rank):
    """Closed form at full size: a cosine mode cos(2 pi k.j / N) is an
    eigenvector of the preconditioner with eigenvalue G(k) (G is even in each
    index), so a sum of modes comes back scaled mode by mode. FP32 and FP64,
    both Hartley implementations (two-stage plans incl. radix 32 at N = 512)."""
    import torch

    ks = [(1, 0, 0), (3, 5, 7), (N // 2, N // 4, 1)]
    amps = [1.0, -0.5, 0.25]
    j = np.arange(N)
    lam = 4 * np.sin(np.pi * j / N) ** 2
    if rank:
        t, w = _oracle_nodes(N, rank)
    pc = sq.sq_precond_setup(N, rank)
    r = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
    zexp = torch.zeros_like(r)
    jj = torch.arange(N, dtype=torch.float64, device="cuda")
    for k, a in zip(ks, amps):
        th = 2 * np.pi * (k[0] * jj[:, None, None] + k[1] * jj[None, :, None] + k[2] * jj[None, None, :]) / N
        mode = a * torch.cos(th)
        g = lam[k[0]] + lam[k[1]] + lam[k[2]]
        G = 1.0 / g if rank == 0 else float(np.sum(np.asarray(w) * np.exp(-np.asarray(t) * g)))
        r += mode
        zexp += G * mode
    for prec, dt, tol in ((sq.SQ_FP64, torch.float64, 1e-12), (sq.SQ_FP32_REFINE, torch.float32, 1e-5)):
        w_ = sq.sq_workspace_create(N, prec)
        for opt in (0, 1):
            try:
                sq.sq_set_option(sq.SQ_OPT_STRIDED_TWO_STAGE, opt)
                z = torch.empty(N ** 3, dtype=dt, device="cuda")
                (sq.sq_apply_precond if dt == torch.float64 else sq.sq_apply_precond_f32)(
                    pc, w_, r.reshape(-1).to(dt).contiguous(), z)
                torch.cuda.synchronize()
            finally:
                sq.sq_set_option(sq.SQ_OPT_STRIDED_TWO_STAGE, 1)
            err = float((z.double().reshape(N, N, N) - zexp).abs().max() / zexp.abs().max())
            assert err <= tol, (prec, opt, err)
        del w_


def test_inner_tolerance_option(sq):
    """SQ_OPT_INNER_TOL_EXP: 2..7 accepted, others rejected; the refined
    solution meets the tolerance at either end of the range."""
    import torch

    for bad in (1, 8):
        with pytest.raises(sq.SqError):
            sq.sq_set_option(sq.SQ_OPT_INNER_TOL_EXP, bad)
    L, n = 4, 8
    N = L * n
    c = sq.sq_build_coeffs(L, n, 5, 0.5, 1.0, 100.0)
    pc = sq.sq_precond_setup(N, 8)
    w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
    psi = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    try:
        for e in (2, 7):
            sq.sq_set_option(sq.SQ_OPT_INNER_TOL_EXP, e)
            info = sq.sq_pcg_solve(c, pc, w, 0, 1e-10, 4000, sq.SQ_FP32_REFINE, None, psi)
            assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-10
    finally:
        sq.sq_set_option(sq.SQ_OPT_INNER_TOL_EXP, 5)


def test_bounded_staging_wait_gives_up_cleanly(sq):
    """Failure detection without a GPU fault: SQ_OPT_WAIT_POLLS = 0 makes the
    FP32 pass E give up on its bulk-copy barrier at once. The kernel falls
    back to global-memory reads, so the solve still reaches the oracle's
    corrector with zero mean and complete info, and reports SQ_ETIMEOUT; the
    next solve with the default limit is clean."""
    re = problem.realization(8, 8, 4, 1.0, 100.0)           # N = 64: two-stage x3 tiles, staged pass E
    c = sq.sq_build_coeffs(8, 8, 4, 0.5, 1.0, 100.0)
    ref = pcg.tight_solve(re.A, re.b[1], re.N)[0]
    try:
        sq.sq_set_option(sq.SQ_OPT_WAIT_POLLS, 0)
        psi, info = _solve(sq, c, re.N, 1, 8, 1e-10, precision=sq.SQ_FP32_REFINE)
    finally:
        sq.sq_set_option(sq.SQ_OPT_WAIT_POLLS, 1 << 22)
    x = _host(psi)
    assert info["status"] == sq.SQ_ETIMEOUT
    assert info["relres_true"] <= 1e-10 and info["iters"] > 0 and info["outer_steps"] >= 1
    assert abs(x.mean()) <= 1e-14 * np.abs(x).max()
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-6
    psi2, info2 = _solve(sq, c, re.N, 1, 8, 1e-10, precision=sq.SQ_FP32_REFINE)
    assert info2["status"] == sq.SQ_OK and info2["relres_true"] <= 1e-10
    assert np.linalg.norm(_host(psi2) - ref) / np.linalg.norm(ref) <= 1e-6


@pytest.mark.slow
def test_full_size_n256_elementwise_against_oracle(sq):
    """The timed configuration solved tight and compared element by element:
    L = 32, n = 8 (N = 256), Bernoulli(1/2) on {1,100}, seed 0, the rank-8
    preconditioner, FP64 PCG to 1e-12 for all three correctors, against the
    oracle's tight solves (run in spawned CPU processes while the GPU works):
    psi within 1e-9 (rel. L2) and A_hom within 1e-10 of its largest entry."""
    import multiprocessing
    import os
    from concurrent.futures import ProcessPoolExecutor

    from tests import oracle_jobs

    L, n, seed = 32, 8, 0
    N = L * n
    workers = max(1, len(os.sched_getaffinity(0)) // 3)
    with ProcessPoolExecutor(max_workers=3, mp_context=multiprocessing.get_context("spawn")) as ex:
        futs = [ex.submit(oracle_jobs.tight_corrector, L, n, seed, 1.0, 100.0, i, workers) for i in range(3)]
        c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
        psis, infos = [], []
        for i in range(3):
            psi, info = _solve(sq, c, N, i, 8, 1e-12)
            psis.append(psi)
            infos.append(info)
        Ah, _ = sq.sq_homogenized_matrix(c, *psis, energy=False)
        refs = [f.result()[0] for f in futs]
    for info in infos:
        assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-12
    for i in range(3):
        x = _host(psis[i])
        assert np.linalg.norm(x - refs[i]) / np.linalg.norm(refs[i]) <= 1e-9, i
    a_edges = assembly.edge_coefficients(rng.cell_values(rng.cell_phases_vec(L, seed), 1.0, 100.0), n)
    Ao = homogenized.ahom_edge(a_edges, [r.reshape(N, N, N) for r in refs])
    assert np.abs(Ah - Ao).max() <= 1e-10 * np.abs(Ao).max()


@pytest.mark.parametrize("N", [16, 48, 96, 256])
@pytest.mark.parametrize("rank", [0, 8])
def test_multiplier_table_and_on_the_fly_agree(sq, N, rank):
    """Pass C reads the tabulated multiplier (N <= 256) or sums it per mode
    (SQ_OPT_MULTIPLIER_TABLE = 0); both give the oracle's preconditioner, in
    FP64 and FP32."""
    import torch

    pc = sq.sq_precond_setup(N, rank)
    G = _core(sq, pc, N, rank)
    for prec, dt, tol in ((sq.SQ_FP64, "float64", 1e-12), (sq.SQ_FP32_REFINE, "float32", 2e-5)):
        w = sq.sq_workspace_create(N, prec)
        r = inputs.random_field(N, 11 * N + rank, np.float64 if dt == "float64" else np.float32)
        ref = precond.apply_precond(G, r.astype(np.float64))
        for opt in (1, 0):
            try:
                sq.sq_set_option(sq.SQ_OPT_MULTIPLIER_TABLE, opt)
                z = torch.empty(N ** 3, dtype=getattr(torch, dt), device="cuda")
                (sq.sq_apply_precond if dt == "float64" else sq.sq_apply_precond_f32)(pc, w, _dev(r.ravel(), dt), z)
                got = _host(z).reshape(N, N, N).astype(np.float64)
            finally:
                sq.sq_set_option(sq.SQ_OPT_MULTIPLIER_TABLE, 1)
            assert _relmax(got, ref) <= tol, (prec, opt)


@pytest.mark.parametrize("P", [8, 16])
def test_fp32_transform_tiles_at_n512(sq, P):
    """N = 512 with 8- and 16-pencil tiles (the latter runs two radix-16
    butterflies per thread in the strided passes' second stage): a sum of
    cosine modes comes back scaled mode by mode by the oracle's multiplier,
    exact and rank 8, through the FP32 transform passes."""
    import torch

    N, rank = 512, 8
    t_, w_ = _oracle_nodes(N, rank)
    lam = 4 * np.sin(np.pi * np.arange(N) / N) ** 2
    ks = [(1, 0, 0), (3, 5, 7), (N // 2, N // 4, 1), (200, 17, 311)]
    amps = [1.0, -0.5, 0.25, 0.125]
    jj = torch.arange(N, dtype=torch.float64, device="cuda")
    for rr in (0, rank):
        pc = sq.sq_precond_setup(N, rr)
        r = torch.zeros((N, N, N), dtype=torch.float64, device="cuda")
        zexp = torch.zeros_like(r)
        for k, a in zip(ks, amps):
            th = 2 * np.pi * (k[0] * jj[:, None, None] + k[1] * jj[None, :, None] + k[2] * jj[None, None, :]) / N
            mode = a * torch.cos(th)
            g = lam[k[0]] + lam[k[1]] + lam[k[2]]
            G = 1.0 / g if rr == 0 else float(np.sum(w_ * np.exp(-t_ * g)))
            r += mode
            zexp += G * mode
        w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
        z = torch.empty(N ** 3, dtype=torch.float32, device="cuda")
        try:
            sq.sq_set_tiles([(N, P, 0, 0)])
            sq.sq_apply_precond_f32(pc, w, r.reshape(-1).float().contiguous(), z)
            torch.cuda.synchronize()
        finally:
            sq.sq_set_tiles([])
        err = float((z.double().reshape(N, N, N) - zexp).abs().max() / zexp.abs().max())
        assert err <= 1e-5, (rr, err)
        del w, z, r, zexp
        torch.cuda.empty_cache()


@pytest.mark.parametrize("Pe", [2, 4, 8, 16])
def test_pass_e_tile_width(sq, Pe):
    """The last pass of the FP32 iteration (x3 transform with x += alpha p,
    p = z + beta p, staging p and x) with its own tile width: the refined
    solve reaches the oracle's corrector for every width."""
    re = problem.realization(8, 8, 6, 1.0, 100.0)
    c = sq.sq_build_coeffs(8, 8, 6, 0.5, 1.0, 100.0)
    ref = pcg.tight_solve(re.A, re.b[2], re.N)[0]
    try:
        sq.sq_set_tiles([(re.N, 16, 0, 0, Pe)])
        psi, info = _solve(sq, c, re.N, 2, 8, 1e-10, precision=sq.SQ_FP32_REFINE)
    finally:
        sq.sq_set_tiles([])
    assert info["status"] == sq.SQ_OK and info["relres_true"] <= 1e-10
    assert np.linalg.norm(_host(psi) - ref) / np.linalg.norm(ref) <= 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_iteration_graphs_match_direct_launches(sq, precision):
    """Single solves replay a CUDA graph of two PCG iterations (SQ_OPT_PCG_GRAPHS
    = 1) or launch every kernel (0): the same kernels with the same parameters,
    so psi, the iteration counts and the number of kernels launched agree
    exactly, for a second output field (a second stored graph) and after an
    option change (a new capture); and the result matches the oracle."""
    import torch

    L, n, seed, rank = 8, 8, 4, 8
    N = L * n
    re = problem.realization(L, n, seed, 1.0, 100.0)
    ref = pcg.tight_solve(re.A, re.b[2], re.N)[0]
    c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
    pc = sq.sq_precond_setup(N, rank)
    w = sq.sq_workspace_create(N, precision)
    outs = {}
    try:
        for mode in (0, 1):
            sq.sq_set_option(sq.SQ_OPT_PCG_GRAPHS, mode)
            runs = []
            for k in range(3):
                if k == 2:  # a new option epoch: the next solve captures again
                    sq.sq_set_option(sq.SQ_OPT_MULTIPLIER_TABLE, 1)
                psi = torch.full((N ** 3,), float(k), dtype=torch.float64, device="cuda")
                l0 = sq.sq_launch_count()
                info = sq.sq_pcg_solve(c, pc, w, 2, 1e-10, 2000, precision, None, psi)
                runs.append((_host(psi), info["iters"], info["status"], sq.sq_launch_count() - l0))
            outs[mode] = runs
    finally:
        sq.sq_set_option(sq.SQ_OPT_PCG_GRAPHS, 1)
    for (x0, it0, st0, l0), (x1, it1, st1, l1) in zip(outs[0], outs[1]):
        assert st0 == st1 == sq.SQ_OK
        assert it0 == it1 and l0 == l1
        assert np.array_equal(x0, x1)
        assert np.linalg.norm(x1 - ref) / np.linalg.norm(ref) <= 1e-6
