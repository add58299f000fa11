"""Oracle jobs for a process pool (spawn context): module-level functions a
child process can import. Each builds its own realization on the CPU, so a
child never touches the GPU; the GPU tests submit them before their own GPU
work and collect the results afterwards."""
import numpy as np


def tight_corrector(L, n, seed, a_lo, a_hi, i, workers=None, tol=1e-13):
    """The oracle's tight solve (exact-preconditioned CG to rel. residual tol,
    zero mean) of corrector i of one realization; returns (psi flat, its)."""
    from oracle import pcg, problem

    re = problem.realization(L, n, seed, a_lo, a_hi)
    x, it, _ = pcg.pcg(re.A, re.b[i], pcg.fft_preconditioner(re.N, 0, workers), tol=tol, maxit=5000)
    return np.ascontiguousarray(x), it
