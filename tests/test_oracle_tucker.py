"""Pins for the paper's Tucker route to the canonical preconditioner
(Sec. 4.2: HOSVD of G+, Tucker-to-canonical) and the 2R + 1 split of
Lemma 4.2."""
import numpy as np
import pytest

from oracle import precond, tucker


@pytest.fixture(scope="module", params=[16, 24])
def g16(request):
    N = request.param
    return N, precond.core_tensor_exact(N)


def test_full_rank_tucker_is_exact(g16):
    N, G = g16
    U, s = tucker.hosvd(G, N)
    assert np.allclose(U.T @ U, np.eye(N), atol=1e-12)
    Gt = tucker.tucker_full(U, tucker.tucker_core(G, U))
    assert np.abs(Gt - G).max() <= 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("r", [3, 5, 8])
def test_hosvd_error_bounds(g16, r):
    # De Lathauwer et al. (2000): sum_{i>r} s_i^2 <= ||G - G_r||_F^2 <= 3 sum_{i>r} s_i^2
    N, G = g16
    U, s = tucker.hosvd(G, r)
    Gt = tucker.tucker_full(U, tucker.tucker_core(G, U))
    err2 = float(((G - Gt) ** 2).sum())
    tail = float((s[r:] ** 2).sum())
    assert tail * (1 - 1e-9) <= err2 <= 3 * tail * (1 + 1e-9)


def test_core_symmetry_and_even_factors(g16):
    N, G = g16
    U, _ = tucker.hosvd(G, 6)
    core = tucker.tucker_core(G, U)
    for perm in ((1, 0, 2), (0, 2, 1), (2, 1, 0)):
        assert np.abs(core - core.transpose(perm)).max() <= 1e-12 * np.abs(core).max()
    # rows k and N - k of the unfolding coincide (lambda_k = lambda_{N-k}),
    # so the leading singular vectors are even
    rev = (-np.arange(N)) % N
    assert np.abs(U - U[rev]).max() <= 1e-10


@pytest.mark.parametrize("r", [4, 7])
def test_tucker_to_canonical_exact_at_zero_tol(g16, r):
    N, G = g16
    U, _ = tucker.hosvd(G, r)
    core = tucker.tucker_core(G, U)
    F1, F2, F3 = tucker.tucker_to_canonical(U, core, 0.0)
    assert F1.shape == (r * r, N)
    Gc = tucker.canonical_full(F1, F2, F3)
    Gt = tucker.tucker_full(U, core)
    assert np.abs(Gc - Gt).max() <= 1e-12 * np.abs(Gt).max()


def test_truncation_lowers_rank_monotonically():
    N = 32
    G = precond.core_tensor_exact(N)
    U, _ = tucker.hosvd(G, 8)
    core = tucker.tucker_core(G, U)
    ranks, errs = [], []
    for tol in (1e-2, 1e-3, 1e-4, 0.0):
        F = tucker.tucker_to_canonical(U, core, tol)
        ranks.append(F[0].shape[0])
        errs.append(tucker.max_relative_error_full(N, tucker.canonical_full(*F)))
    assert ranks == sorted(ranks) and ranks[-1] == 64
    assert errs[-1] < 1e-3 and errs[0] > errs[-1]


@pytest.mark.parametrize("N,R", [(16, 4), (24, 6), (32, 8)])
def test_lemma_split_is_the_projected_exponential_sum(N, R):
    # the 2R + 1 terms of Lemma 4.2 reproduce the exponential sum on every
    # nonzero mode and vanish at the zero mode, exactly as G_R with its
    # (0,0,0) entry set to 0 (what the mean projection does to the R-term
    # tensor); the error on the nonzero modes is that of the R-term sum
    t, w = precond.rank_r_nodes(N, R)
    F1, F2, F3 = tucker.lemma_split(N, t, w)
    assert F1.shape == (2 * R + 1, N)
    Gs = tucker.canonical_full(F1, F2, F3)
    Ge = precond.core_tensor_from_nodes(N, t, w)
    assert abs(Gs[0, 0, 0]) <= 1e-12 * np.abs(Ge).max()
    assert np.abs(Gs - Ge).max() <= 1e-12 * np.abs(Ge).max()
    assert abs(tucker.max_relative_error_full(N, Gs) - precond.max_relative_error(N, t, w)) <= 1e-9
