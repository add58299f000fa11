"""CG / PCG on the zero-mean subspace and the reference solves (Sec. 4.1).

Test infrastructure only (see ``oracle/__init__``).

The paper solves B^+ A u = B^+ f on <u, 1> = 0 (Eqs. 24-25) with Matlab's
``pcg``. This oracle writes the same Hestenes-Stiefel recurrence:

    x0 = 0, r0 = b, z0 = P r0, p0 = z0
    q = A p, alpha = (r.z)/(p.q), x += alpha p, r -= alpha q,
    z = P r, beta = (r.z)_new/(r.z)_old, p = z + beta p

and Matlab's stopping rule: ||b - A x||_2 / ||b||_2 <= tol, tested on the
recurrence residual and confirmed on the true residual (iteration continues
while the true residual fails). The iteration count is the number of x
updates. The solution is finally projected to zero mean (the corrector is
defined up to a constant; Sec. 4.1 works on <u, 1> = 0).
"""
from __future__ import annotations

import numpy as np

from . import precond as _pc


def pcg(A, b: np.ndarray, apply_P=None, tol: float = 1e-10, maxit: int = 10000, x0=None):
    """Returns (x, iterations, true relative residual). ``apply_P`` maps a flat
    residual to a flat preconditioned residual (None = plain CG)."""
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    z = r.copy() if apply_P is None else apply_P(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    relres = np.linalg.norm(r) / nb
    while it < maxit:
        if relres <= tol:
            true_rel = np.linalg.norm(b - A @ x) / nb
            if true_rel <= tol:
                break
        q = A @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        relres = np.linalg.norm(r) / nb
        z = r.copy() if apply_P is None else apply_P(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    x -= x.mean()
    return x, it, float(np.linalg.norm(b - A @ x) / nb)


def fft_preconditioner(N: int, rank: int, workers: int | None = None):
    """Flat-vector wrapper of the Sec. 4.2 preconditioner (exact if rank == 0);
    workers: FFT threads (None = numpy's single-threaded FFT)."""
    G = _pc.core_tensor(N, rank)

    def apply(r):
        return _pc.apply_precond(G, r.reshape(N, N, N), workers).ravel()

    return apply


def tight_solve(A, b: np.ndarray, N: int, tol: float = 1e-13):
    """The plain definition of the discrete corrector: the zero-mean solution of
    A psi = b, reached by exact-preconditioned CG to rel. residual ``tol``."""
    x, it, rel = pcg(A, b, fft_preconditioner(N, 0), tol=tol, maxit=5000)
    return x, it, rel


def dense_solve(A, b: np.ndarray) -> np.ndarray:
    """Minimum-norm least-squares solution (zero mean, since ker A = span{1})."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    x = np.linalg.lstsq(Ad, b, rcond=None)[0]
    return x - x.mean()
