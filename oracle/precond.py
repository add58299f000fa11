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
* A second exponential sum, :func:`lsq_nodes`: geometric nodes with weights
  fitted by least squares to the relative error over a log-uniform sample of
  the discrete spectrum, kept only where it beats the trapezoid rule. It is
  the rank-R construction the GPU library uses, written here independently in
  numpy; it is pinned by positivity, by the least-squares normal equations,
  by beating the trapezoid rule on every eigenvalue, and by its convergence
  to 1/x as R grows (tests/test_oracle_precond).
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


def rank_r_nodes(N: int, R: int, dim: int = 3):
    """Quadrature nodes t_r and weights w_r of the exponential sum (R >= 2).

    Trapezoid rule for 1/x = int exp(s - x e^s) ds on x in [lambda_min, X]
    (X = 4 dim, the largest eigenvalue of the dim-dimensional periodic
    Laplacian: 12 in 3D) with three error sources balanced at one level eps:
      lower truncation  ~ X e^{s_lo}             -> s_lo = ln(eps / X)
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
        s_lo = le - math.log(4.0 * dim)
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


def spectrum_values(N: int, dim: int = 3) -> np.ndarray:
    """The distinct nonzero eigenvalues of the dim-dimensional periodic
    Laplacian, l_i + l_j (+ l_k), sorted ascending. Values within a relative
    1e-12 of the last kept value count as one (equal sums of different index
    triples differ only by rounding)."""
    lam = laplacian_eigenvalues(N)[: N // 2 + 1]   # l_k = l_{N-k}: half the range holds every value
    if dim == 2:
        g = lam[:, None] + lam[None, :]
    else:
        g = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    g = np.sort(g.ravel())
    g = g[g > 0.0]
    keep = [g[0]]
    for x in g[1:]:
        if x > keep[-1] * (1.0 + 1e-12):
            keep.append(x)
    return np.array(keep)


def log_uniform_sample(values: np.ndarray, K: int = 3000) -> np.ndarray:
    """For each of K points of the geometric grid from values[0] to
    values[-1], the nearest of the given (sorted, distinct) values; repeats
    dropped, ascending."""
    x0, x1 = values[0], values[-1]
    out = []
    for m in range(K):
        target = x0 * (x1 / x0) ** (m / (K - 1))
        i = int(np.searchsorted(values, target))
        hi = values[min(i, len(values) - 1)]
        lo = values[i - 1] if i > 0 else hi
        pick = lo if (i > 0 and (i == len(values) or abs(lo - target) < abs(hi - target))) else hi
        if not out or pick > out[-1]:
            out.append(pick)
    return np.array(out)


def sampled_relative_error(x: np.ndarray, t, w) -> float:
    """max over the values x of |x * sum_r w_r exp(-t_r x) - 1|."""
    g = np.exp(-np.outer(x, np.asarray(t, dtype=np.float64))) @ np.asarray(w, dtype=np.float64)
    return float(np.abs(x * g - 1.0).max())


def lsq_nodes(N: int, R: int, dim: int = 3):
    """Exponential sum for 1/x with geometric nodes and least-squares weights
    (our reading of the rank-R construction; the paper states the Laplace
    transform route of Eq. 34 and leaves the nodes open). Returns (t, w).

    1. x ranges over the distinct nonzero Laplacian eigenvalues
       (:func:`spectrum_values`), sampled log-uniformly at 3000 points
       (:func:`log_uniform_sample`).
    2. For each (a, b) on a grid, a in -ln(4 dim) - 6 + 7 i/(g-1) and
       b in ln(1/lambda_min) - 1 + 5 j/(g-1) (g = 40 for R <= 16, else 20),
       the nodes are t_r = exp(a + (b - a) r/(R-1)) and the weights solve
       min_w || x exp(-x t) w - 1 ||_2 over the sample (numpy lstsq).
    3. Fits with any w_r <= 0 are discarded (G_R must stay positive), and so
       are numerically singular ones: the largest |diagonal entry| of the
       triangular factor of a QR decomposition of the sample matrix above
       1e10 times the smallest (many terms over a narrow spectrum, where the
       weights would be rounding noise). Of the rest the one with the
       smallest largest sampled error is kept (the first in (i, j) order on
       ties).
    4. The fit replaces the trapezoid rule (:func:`rank_r_nodes`) only if its
       largest error over every distinct eigenvalue is smaller; for R > 32,
       or with fewer than 2R sample points, the trapezoid rule is returned.
    """
    t_trap, w_trap = rank_r_nodes(N, R, dim)
    if R > 32:
        return t_trap, w_trap
    values = spectrum_values(N, dim)
    x = log_uniform_sample(values)
    if len(x) < 2 * R:
        return t_trap, w_trap
    lam_min = 4.0 * math.sin(math.pi / N) ** 2
    g = 40 if R <= 16 else 20
    best, best_t, best_w = np.inf, None, None
    for i in range(g):
        a = -math.log(4.0 * dim) - 6.0 + 7.0 * i / (g - 1)
        for j in range(g):
            b = math.log(1.0 / lam_min) - 1.0 + 5.0 * j / (g - 1)
            t = np.exp(a + (b - a) * np.arange(R) / (R - 1))
            E = x[:, None] * np.exp(-np.outer(x, t))
            d = np.abs(np.diag(np.linalg.qr(E, mode="r")))
            if not d.min() > 0.0 or d.max() > 1e10 * d.min():
                continue
            w = np.linalg.lstsq(E, np.ones(len(x)), rcond=None)[0]
            if not np.all(w > 0.0):
                continue
            err = float(np.abs(E @ w - 1.0).max())
            if err < best:
                best, best_t, best_w = err, t, w
    if best_t is not None and sampled_relative_error(values, best_t, best_w) < sampled_relative_error(
            values, t_trap, w_trap):
        return best_t, best_w
    return t_trap, w_trap


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


def apply_precond(G: np.ndarray, r: np.ndarray, workers: int | None = None) -> np.ndarray:
    """z = F^{-1} (G * F r) on an (N,N,N) field (Eq. 31); zero-mean output.
    workers: threads of the FFT (scipy.fft); None = numpy's single-threaded FFT."""
    if workers is None:
        return np.real(np.fft.ifftn(G * np.fft.fftn(r)))
    import scipy.fft

    return np.real(scipy.fft.ifftn(G * scipy.fft.fftn(r, workers=workers), workers=workers))


def spectral_ratio(N: int, R: int) -> float:
    """max/min over nonzero modes of g * G_R (1 for the exact tensor)."""
    lam = laplacian_eigenvalues(N)
    g = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    G = core_tensor_rank_r(N, R)
    m = g > 0
    prod = g[m] * G[m]
    return float(prod.max() / prod.min())
