"""Pins for the oracle's ensemble statistics (Sec. 5, Eq. A_hom_Empir and the
sample standard deviation sigma^M_L)."""
import numpy as np
import pytest

from oracle import ensemble


def test_stats_of_a_worked_example():
    # A^(1) = I, A^(2) = 10 I: mean 5.5 I; sigma = sqrt(2 * 4.5^2 / 1) = 4.5 sqrt(2) on the diagonal
    mean, sigma = ensemble.ensemble_stats([np.eye(3), 10 * np.eye(3)])
    assert np.allclose(mean, 5.5 * np.eye(3), rtol=0, atol=1e-15)
    assert np.allclose(sigma, 4.5 * np.sqrt(2.0) * np.eye(3), rtol=1e-15, atol=0)


def test_stats_of_three_scalars_by_hand():
    # entries 1, 2, 6: mean 3, deviations -2, -1, 3, sum of squares 14, sigma sqrt(7)
    A = [np.full((3, 3), v) for v in (1.0, 2.0, 6.0)]
    mean, sigma = ensemble.ensemble_stats(A)
    assert np.allclose(mean, 3.0) and np.allclose(sigma, np.sqrt(7.0))


def test_stats_need_two_realizations():
    with pytest.raises(ValueError):
        ensemble.ensemble_stats([np.eye(3)])


def test_constant_coefficient_ensemble_is_deterministic():
    # p_hi = 0: every cell a_lo, the correctors vanish and A_hom = a_lo I exactly
    mean, sigma, As = ensemble.ensemble_ahom(2, 4, [3, 4, 5], 2.5, 7.0, p_hi=0.0)
    assert np.allclose(As, 2.5 * np.eye(3), rtol=0, atol=1e-13)
    assert np.allclose(mean, 2.5 * np.eye(3), rtol=0, atol=1e-13) and np.abs(sigma).max() < 1e-13


def test_random_ensemble_bounds_and_spread():
    # per realization: a_lo <= A_ii <= mean of its edge coefficients a_i (the
    # energy with psi = 0 as the competitor); the ensemble spread is positive
    from oracle import problem

    lo, hi = 1.0, 10.0
    seeds = list(range(4))
    mean, sigma, As = ensemble.ensemble_ahom(3, 2, seeds, lo, hi)
    for s, A in zip(seeds, As):
        a = problem.realization(3, 2, s, lo, hi).a_edges
        for i in range(3):
            assert lo - 1e-12 <= A[i, i] <= a[i].mean() + 1e-12
        assert np.abs(A - A.T).max() <= 1e-10 * np.abs(A).max()
    assert np.all(sigma >= 0) and sigma[0, 0] > 0
    assert np.allclose(mean, As.mean(axis=0), rtol=1e-15, atol=0)
