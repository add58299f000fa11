"""Spectral preconditioner: pseudo-inverse of the periodic Laplacian (Sec. 4).

Test infrastructure only (see ``oracle/__init__``).

* Eigenvalues (Eqs. 28-29): the 1D periodic Laplacian is the circulant matrix
  with first column p = (2, -1, 0, ..., 0, -1); its eigenvalues are the DFT of
  p, lambda_k = [F p]_k = 2 - 2 cos(2 pi k / N) (real, lambda_0 = 0). The
  paper prints the circulant with mixed signs (Eqs. 12-13); this oracle takes
  the positive semidefinite form.
* Core tensor (Eqs. 32-33): G+(k1,k2,k3) = 1 / (lambda_k1 + lambda_k2 +
  lambda_k3) with G+(0,0,0) = 0 (pseudo-inverse on the zero-mean subspace).
  The prefactor (1+lambda)/2 and delta of Sec. 4.1 are taken as 1 and 0; a
  positive scalar on the preconditioner leaves the PCG iterates unchanged.
* Rank-R canonical approximation (Eq. 34, Lemma 4.2). The paper proves
  existence through the Laplace transform 1/x = int_0^inf exp(-x t) dt (the
  printed 1/pi prefactor is dropped: the integral is exactly 1/x) and builds
  its factors by multigrid Tucker + Tucker-to-canonical, an algorithm it does
  not state (``oracle/tucker`` takes that route with the plain HOSVD and a
  core-slice Tucker-to-canonical). This module follows the Laplace-transform
  route: substitute
  t = e^s, so 1/x = int_R exp(s - x e^s) ds, and apply the trapezoid (sinc)
  rule on R equispaced nodes s_r. Because exp(-t x) with x = l1 + l2 + l3
  factorises, G_R(k1,k2,k3) = sum_r u_r(k1) u_r(k2) u_r(k3) with
  u_r(k) = w_r^(1/3) exp(-t_r lambda_k), t_r = e^{s_r}, w_r = eta e^{s_r}.
  The node interval and step balance the truncation and step errors at one
  level (see :func:`rank_r_nodes`); x ranges over [lambda_min, 12] with
  lambda_min = 4 sin^2(pi/N). All w_r > 0, so G_R is positive on every
  nonzero mode. The node placement is a reading of ours (the paper gives
  none); the quadrature is pinned by its convergence to the exact G+ as R
  grows.
* Apply (Eq. 31): z = F^{-1} diag(G) F r with the 3D DFT (numpy), DC := 0.
"""
from __future__ import annotations

import math

import numpy as np


def laplacian_eigenvalues_fft(N: int) -> np.ndarray:
    """lambda_k = [F p]_k, the DFT of the circulant's first column (Eq. 29)."""
    p = np.zeros(N)
    p[0] = 2.0
    p[1] -= 1.0
    p[-1] -= 1.0
    return np.fft.fft(p).real


def laplacian_eigenvalues(N: int) -> np.ndarray:
    """Closed form of the same eigenvalues: 4 sin^2(pi k / N)."""
    k = np.arange(N)
    return 4.0 * np.sin(np.pi * k / N) ** 2


def core_tensor_exact(N: int) -> np.ndarray:
    """G+(k1,k2,k3) = 1/(l1+l2+l3), G+(0,0,0) = 0 (Eq. 33)."""
    lam = laplacian_eigenvalues_fft(N)
    g = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    G = np.zeros_like(g)
    nz = g > 0
    G[nz] = 1.0 / g[nz]
    return G


def rank_r_nodes(N: int, R: int):
    """Quadrature nodes t_r and weights w_r of the exponential sum (R >= 2).

    Trapezoid rule for 1/x = int exp(s - x e^s) ds on x in [lambda_min, 12]
    with three error sources balanced at one level eps:
      lower truncation  ~ 12 e^{s_lo}            -> s_lo = ln(eps / 12)
      upper truncation  ~ exp(-lambda_min e^{s_hi}) -> s_hi = ln(ln(1/eps) / lambda_min)
      step error        ~ exp(-pi^2 / eta)       (integrand analytic in the
                                                  strip |Im s| < pi/2)
    with eta = (s_hi - s_lo)/(R - 1). eps is found by bisection on ln(eps)
    (200 halvings of [ln 1e-300, ln 0.5]).
    """
    if R < 2:
        raise ValueError("rank R must be >= 2")
    lam_min = 4.0 * math.sin(math.pi / N) ** 2

    def interval(le):
        eps = math.exp(le)
        s_lo = le - math.log(12.0)
        s_hi = math.log(-le / lam_min)
        return s_lo, s_hi, (s_hi - s_lo) / (R - 1), eps

    lo, hi = math.log(1e-300), math.log(0.5)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        _, _, eta, eps = interval(mid)
        if math.exp(-math.pi ** 2 / eta) > eps:
            lo = mid   # step error dominates: a larger eps is consistent
        else:
            hi = mid
    s_lo, _, eta, _ = interval(0.5 * (lo + hi))
    s = s_lo + eta * np.arange(R)
    return np.exp(s), eta * np.exp(s)


def rank_r_factors(N: int, R: int) -> np.ndarray:
    """Canonical factors u_r(k), shape (R, N); the same vector serves all three
    axes because the grid is cubic."""
    t, w = rank_r_nodes(N, R)
    lam = laplacian_eigenvalues(N)
    return np.cbrt(w)[:, None] * np.exp(-t[:, None] * lam[None, :])


def core_tensor_rank_r(N: int, R: int) -> np.ndarray:
    """G_R = sum_r u_r (x) u_r (x) u_r with G_R(0,0,0) := 0."""
    U = rank_r_factors(N, R)
    G = np.einsum("ri,rj,rk->ijk", U, U, U)
    G[0, 0, 0] = 0.0
    return G


def core_tensor_from_nodes(N: int, t, w) -> np.ndarray:
    """G(k) = sum_r w_r exp(-t_r (l_k1 + l_k2 + l_k3)), G(0,0,0) := 0, for given
    nodes t_r and weights w_r (an exponential sum for 1/x, Eq. 34)."""
    lam = laplacian_eigenvalues(N)
    U = np.cbrt(np.asarray(w, dtype=np.float64))[:, None] * np.exp(-np.outer(np.asarray(t, dtype=np.float64), lam))
    G = np.einsum("ri,rj,rk->ijk", U, U, U)
    G[0, 0, 0] = 0.0
    return G


def max_relative_error(N: int, t, w) -> float:
    """max over nonzero modes of |g * G(g) - 1| for the exponential sum (t, w)."""
    lam = laplacian_eigenvalues(N)
    g = np.unique(np.round((lam[:, None, None] + lam[None, :, None] + lam[None, None, :]).ravel(), 13))
    g = g[g > 0]
    G = np.exp(-np.outer(g, np.asarray(t, dtype=np.float64))) @ np.asarray(w, dtype=np.float64)
    return float(np.abs(g * G - 1.0).max())


def core_tensor(N: int, rank: int) -> np.ndarray:
    """rank 0 = exact Fourier diagonal, else the rank-R canonical tensor."""
    return core_tensor_exact(N) if rank == 0 else core_tensor_rank_r(N, rank)


def apply_precond(G: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z = F^{-1} (G * F r) on an (N,N,N) field (Eq. 31); zero-mean output."""
    return np.real(np.fft.ifftn(G * np.fft.fftn(r)))


def spectral_ratio(N: int, R: int) -> float:
    """max/min over nonzero modes of g * G_R (1 for the exact tensor)."""
    lam = laplacian_eigenvalues(N)
    g = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    G = core_tensor_rank_r(N, R)
    m = g > 0
    prod = g[m] * G[m]
    return float(prod.max() / prod.min())
