"""Batched solves (one launch per kernel for a mixed-size batch) against the
oracle and against single solves of the same precision scheme."""
import numpy as np
import pytest

from oracle import pcg, problem

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


def _empty(N):
    import torch

    return torch.empty(N ** 3, dtype=torch.float64, device="cuda")


def test_mixed_size_batch_matches_oracle(sq):
    # two realizations of different grid size (N = 16 and 24), three RHS each
    cases = [(4, 4, 3, 1.0, 10.0), (6, 4, 5, 1.0, 100.0)]
    precs = {}
    descs, pl, refs = [], [], []
    for L, n, seed, lo, hi in cases:
        N = L * n
        c = sq.sq_build_coeffs(L, n, seed, 0.5, lo, hi)
        precs.setdefault(N, sq.sq_precond_setup(N, 0))
        re = problem.realization(L, n, seed, lo, hi)
        for i in range(3):
            descs.append((c, i, _empty(N)))
            pl.append(precs[N])
            refs.append(pcg.tight_solve(re.A, re.b[i], N)[0])
    b = sq.sq_batch_create(descs, pl)
    infos = sq.sq_pcg_solve_batched(b, 1e-10, 2000)
    for (c, i, psi), ref, inf in zip(descs, refs, infos):
        assert inf["status"] == sq.SQ_OK and inf["relres_true"] <= 1e-10, inf
        x = psi.cpu().numpy()
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-6
        assert abs(x.mean()) <= 1e-12 * np.abs(x).max()
    # a second solve of the same batch (graph replay, scalars reset) gives the same result
    first = [psi.cpu().numpy().copy() for _, _, psi in descs]
    infos2 = sq.sq_pcg_solve_batched(b, 1e-10, 2000)
    for (c, i, psi), x1, i1, i2 in zip(descs, first, infos, infos2):
        assert np.array_equal(psi.cpu().numpy(), x1) and i1["iters"] == i2["iters"]
    # with the kernel-event profile on, the graph's launches run one by one:
    # the same result, and the profile sees 6 inner launches per iteration
    sq.sq_profile_enable(True)
    try:
        infos3 = sq.sq_pcg_solve_batched(b, 1e-10, 2000)
        prof = sq.sq_profile_read()
    finally:
        sq.sq_profile_enable(False)
    for (c, i, psi), x1, i1, i3 in zip(descs, first, infos, infos3):
        assert np.array_equal(psi.cpu().numpy(), x1) and i1["iters"] == i3["iters"]
    ms, nl = prof["batch_inner"]
    loop_ms, nloop = prof["batch_inner_loop"]
    assert nl > 0 and nl % 6 == 0 and 0 < ms <= loop_ms and nloop == infos3[0]["outer_steps"]


def test_batch_matches_single_solves(sq):
    L, n = 8, 4
    N = L * n
    pc = sq.sq_precond_setup(N, 8)
    w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
    descs, singles = [], []
    for seed in range(3):
        c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 10.0)
        for i in range(3):
            descs.append((c, i, _empty(N)))
            ps = _empty(N)
            sq.sq_pcg_solve(c, pc, w, i, 1e-8, 2000, sq.SQ_FP32_REFINE, None, ps)
            singles.append(ps.cpu().numpy())
    b = sq.sq_batch_create(descs, [pc] * len(descs), tiles=[(N, 4, 8)])
    infos = sq.sq_pcg_solve_batched(b, 1e-8, 2000)
    for (c, i, psi), xs, inf in zip(descs, singles, infos):
        assert inf["status"] == sq.SQ_OK and inf["relres_true"] <= 1e-8
        x = psi.cpu().numpy()
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-6


def test_batch_degenerate_and_invalid(sq):
    c0 = sq.sq_build_coeffs(4, 4, 0, 0.5, 2.0, 2.0)    # constant coefficient: b = 0
    c1 = sq.sq_build_coeffs(4, 4, 1, 0.5, 1.0, 10.0)
    pc = sq.sq_precond_setup(16, 0)
    descs = [(c0, 0, _empty(16)), (c1, 1, _empty(16))]
    infos = sq.sq_pcg_solve_batched(sq.sq_batch_create(descs, [pc, pc]), 1e-8, 500)
    assert infos[0]["status"] == sq.SQ_OK and infos[0]["iters"] == 0
    assert np.abs(descs[0][2].cpu().numpy()).max() == 0.0
    assert infos[1]["status"] == sq.SQ_OK
    with pytest.raises(sq.SqError):
        sq.sq_batch_create([(c1, 0, _empty(16))], [sq.sq_precond_setup(32, 0)])   # N mismatch
    with pytest.raises(sq.SqError):
        sq.sq_batch_create([(c1, 0, _empty(16))], [pc], tiles=[(16, 3, 4)])       # P not a power of two


def test_batch_two_stage_tiles_mixed_sizes(sq):
    """Default tiles (P = 16, 8, 16, 16 for N = 32, 48, 64, 96) take the two-stage
    Hartley tiles inside the batched kernels, radix-3 and radix-6 plans included:
    the batch matches the oracle (N = 32, 48) and single solves (all sizes)."""
    import torch

    cases = [(8, 4, 41), (12, 4, 42), (16, 4, 43), (24, 4, 44)]
    descs, pl, singles, refs = [], [], [], []
    for L, n, seed in cases:
        N = L * n
        c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 10.0)
        pc = sq.sq_precond_setup(N, 0)
        w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
        ps = _empty(N)
        sq.sq_pcg_solve(c, pc, w, 1, 1e-9, 2000, sq.SQ_FP32_REFINE, None, ps)
        singles.append(ps.cpu().numpy())
        descs.append((c, 1, _empty(N)))
        pl.append(pc)
        if N <= 48:
            re = problem.realization(L, n, seed, 1.0, 10.0)
            refs.append(pcg.tight_solve(re.A, re.b[1], N)[0])
        else:
            refs.append(None)
    infos = sq.sq_pcg_solve_batched(sq.sq_batch_create(descs, pl), 1e-9, 2000)
    torch.cuda.synchronize()
    for (c, i, psi), xs, ref, inf in zip(descs, singles, refs, infos):
        assert inf["status"] == sq.SQ_OK and inf["relres_true"] <= 1e-9
        x = psi.cpu().numpy()
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-6
        if ref is not None:
            assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-6


def test_batch_two_stage_tiles_rank8(sq):
    """Rank-8 preconditioner with default tiles: the batched pass C takes the
    two-stage tile with the runtime-rank multiplier; the batch matches single
    solves of the same preconditioner."""
    import torch

    descs, pl, singles = [], [], []
    for L, n, seed in [(8, 4, 51), (16, 4, 52), (24, 4, 53)]:
        N = L * n
        c = sq.sq_build_coeffs(L, n, seed, 0.5, 1.0, 100.0)
        pc = sq.sq_precond_setup(N, 8)
        w = sq.sq_workspace_create(N, sq.SQ_FP32_REFINE)
        for i in (0, 2):
            ps = _empty(N)
            sq.sq_pcg_solve(c, pc, w, i, 1e-9, 3000, sq.SQ_FP32_REFINE, None, ps)
            singles.append(ps.cpu().numpy())
            descs.append((c, i, _empty(N)))
            pl.append(pc)
    infos = sq.sq_pcg_solve_batched(sq.sq_batch_create(descs, pl), 1e-9, 3000)
    torch.cuda.synchronize()
    for (c, i, psi), xs, inf in zip(descs, singles, infos):
        assert inf["status"] == sq.SQ_OK and inf["relres_true"] <= 1e-9
        x = psi.cpu().numpy()
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-6
