"""The no-allocation A_hom entry point against the regular one.

sq_homogenized_matrix_noalloc exists for callers that may not allocate device
memory when they need the result (stream capture, framework-owned memory
pools). It must give the same matrix as sq_homogenized_matrix on the same
inputs, on repeated calls that reuse its fixed scratch array. This file is
collected last so a run that stops at the first failure has run every other
test before it; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

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


def _case(sq, L, n, seed, a_lo, a_hi):
    import torch

    N = L * n
    phase = (np.random.default_rng(seed).random(L ** 3) < 0.5).astype(np.uint8)
    c = sq.sq_coeffs_from_host(L, n, phase, a_lo, a_hi)
    psis = [torch.from_numpy(inputs.random_field(N, seed + i).ravel()).cuda() for i in range(3)]
    A_ref, E_ref = sq.sq_homogenized_matrix(c, *psis)
    d_phase = torch.from_numpy(phase).cuda()
    return d_phase, psis, A_ref, E_ref


def test_noalloc_matches_regular_entry_point_twice(sq):
    import torch

    cases = [(4, 4, 11, 1.0, 10.0), (6, 8, 12, 1.0, 100.0)]
    out = torch.full((18,), float("nan"), dtype=torch.float64, device="cuda")
    for L, n, seed, a_lo, a_hi in cases:      # two calls in a row on the shared scratch
        d_phase, psis, A_ref, E_ref = _case(sq, L, n, seed, a_lo, a_hi)
        sq.sq_homogenized_matrix_noalloc(L, n, d_phase, a_lo, a_hi, *psis, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        scale = np.abs(A_ref).max()
        assert np.abs(got[:9].reshape(3, 3) - A_ref).max() <= 1e-12 * scale
        assert np.abs(got[9:].reshape(3, 3) - E_ref).max() <= 1e-12 * scale


def test_noalloc_rejects_oversized_grid(sq):
    import torch

    phase = torch.zeros(1, dtype=torch.uint8, device="cuda")
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(18, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SqError) as e:
        sq.sq_homogenized_matrix_noalloc(128, 8, phase, 1.0, 10.0, f, f, f, out)   # N = 1024 > 512
    assert e.value.status == sq.SQ_EINVAL


@pytest.mark.parametrize("a_lo,a_hi", [(float("inf"), 10.0), (1.0, float("inf"))])
def test_noalloc_rejects_infinite_coefficient(sq, a_lo, a_hi):
    import torch

    phase = torch.zeros(64, dtype=torch.uint8, device="cuda")
    f = torch.zeros(16 ** 3, dtype=torch.float64, device="cuda")
    out = torch.zeros(18, dtype=torch.float64, device="cuda")
    with pytest.raises(sq.SqError) as e:
        sq.sq_homogenized_matrix_noalloc(4, 4, phase, a_lo, a_hi, f, f, f, out)
    assert e.value.status == sq.SQ_EINVAL
