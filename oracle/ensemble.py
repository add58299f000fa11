"""Ensemble statistics of the homogenized matrix over M realizations of the
random checkerboard at a fixed period L (Sec. 5, "Example of application to
numerical estimation of the homogenized coefficient matrix"):

  empirical average    A^M_L = (1/M) sum_m A^(m)_L            (Eq. A_hom_Empir)
  standard deviation   sigma^M_L = sqrt( sum_m (A^(m)_L - A^M_L)^2 / (M-1) )

entry-wise, the computable estimate of sigma_L in Eq. var (which bounds it by
C L^{-d/2}). A^(m)_L is the edge-form A_hom of realization m (Eq. 21 on the
grid), from tight solves of the three correctors.

Test infrastructure only (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from . import homogenized, pcg, problem


def ensemble_stats(A_list):
    """(mean, sigma) entry-wise over M >= 2 matrices: the two formulas above,
    summed in the order given."""
    A = np.asarray(A_list, dtype=np.float64)
    M = A.shape[0]
    if M < 2:
        raise ValueError("the standard deviation needs M >= 2 realizations")
    mean = np.zeros(A.shape[1:])
    for m in range(M):
        mean += A[m]
    mean /= M
    ss = np.zeros(A.shape[1:])
    for m in range(M):
        d = A[m] - mean
        ss += d * d
    return mean, np.sqrt(ss / (M - 1))


def realization_ahom(L: int, n: int, seed: int, a_lo: float, a_hi: float, p_hi: float = 0.5):
    """Edge-form A_hom of one realization from tight solves (rel. residual 1e-13)."""
    re = problem.realization(L, n, seed, a_lo, a_hi, p_hi)
    psis = [pcg.tight_solve(re.A, re.b[i], re.N)[0].reshape(re.N, re.N, re.N) for i in range(3)]
    return homogenized.ahom_edge(re.a_edges, psis)


def ensemble_ahom(L: int, n: int, seeds, a_lo: float, a_hi: float, p_hi: float = 0.5):
    """(mean, sigma, per-realization matrices) over the given seeds."""
    As = np.array([realization_ahom(L, n, s, a_lo, a_hi, p_hi) for s in seeds])
    mean, sigma = ensemble_stats(As)
    return mean, sigma, As
