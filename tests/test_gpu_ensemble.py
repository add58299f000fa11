"""Ensemble statistics of A_hom through the C ABI (sq_ensemble_ahom) against
the oracle (Sec. 5: empirical average and sample standard deviation over M
realizations), plus the L^{-3/2} decay of the spread (Eq. var, d = 3)."""
import numpy as np
import pytest

from oracle import ensemble

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


@pytest.mark.parametrize("rank", [0, 6])
def test_ensemble_matches_oracle(sq, rank):
    L, n, seeds, lo, hi = 4, 4, [11, 12, 13, 14, 15, 16], 1.0, 10.0
    mo, so, Ao = ensemble.ensemble_ahom(L, n, seeds, lo, hi)
    r = sq.sq_ensemble_ahom(L, n, seeds, 0.5, lo, hi, rank=rank, tol=1e-11, max_iter=3000)
    assert r["status"] == sq.SQ_OK
    scale = np.abs(Ao).max()
    assert np.abs(r["per_realization"] - Ao).max() <= 1e-9 * scale
    assert np.abs(r["mean"] - mo).max() <= 1e-9 * scale
    assert np.abs(r["sigma"] - so).max() <= 1e-8 * scale
    assert r["iters"].shape == (6, 3) and r["iters"].min() > 0


def test_chunking_does_not_change_results(sq):
    seeds = list(range(20, 27))
    a = sq.sq_ensemble_ahom(6, 4, seeds, 0.5, 1.0, 100.0, tol=1e-10)
    b = sq.sq_ensemble_ahom(6, 4, seeds, 0.5, 1.0, 100.0, tol=1e-10, chunk=3)
    assert np.abs(a["per_realization"] - b["per_realization"]).max() <= 1e-12 * np.abs(a["mean"]).max()
    assert np.allclose(a["sigma"], b["sigma"], rtol=1e-9, atol=1e-14)


def test_constant_coefficient_ensemble(sq):
    r = sq.sq_ensemble_ahom(4, 4, [1, 2, 3], 0.0, 2.5, 7.0)
    assert np.allclose(r["mean"], 2.5 * np.eye(3), rtol=0, atol=1e-13)
    assert np.abs(r["sigma"]).max() <= 1e-13


def test_invalid_arguments(sq):
    with pytest.raises(sq.SqError):
        sq.sq_ensemble_ahom(4, 4, [1], 0.5, 1.0, 10.0)          # M < 2
    with pytest.raises(sq.SqError):
        sq.sq_ensemble_ahom(5, 4, [1, 2], 0.5, 1.0, 10.0)       # N = 20 is not 2^a 3^b


def test_spread_decays_like_l_to_minus_three_halves(sq):
    """sigma_L <= C L^{-3/2} (Eq. var): the fitted exponent of the diagonal
    spread over L = 4, 8, 16 (n = 4, 24 fixed seeds each) lies near -3/2."""
    Ls = [4, 8, 16]
    sig = []
    for L in Ls:
        r = sq.sq_ensemble_ahom(L, 4, list(range(1000, 1024)), 0.5, 1.0, 10.0, tol=1e-8)
        assert r["status"] == sq.SQ_OK
        sig.append(np.mean(np.diag(r["sigma"])))
    slope = np.polyfit(np.log(Ls), np.log(sig), 1)[0]
    assert -2.2 <= slope <= -0.8, (sig, slope)
