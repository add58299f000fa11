"""Independent 2D cell-centred scheme, used only to pin the node scheme.

Test infrastructure only (see ``oracle/__init__``).

In 2D the homogenized matrix obeys Keller's duality: for a field sigma and its
reciprocal, A[sigma] R A[1/sigma] R^T = I with R the 90-degree rotation. The
discrete node scheme of Sec. 3 (edge conductance = mean of the two voxels
beside the edge) has an exact discrete dual: unknowns at voxel centres,
conductance between neighbouring voxels = harmonic mean of their values. The
dual edge crossing a primal edge then carries the reciprocal conductance, so
the duality holds to rounding for any periodic voxel field. For the
two-phase checkerboard this gives A_node * A_vox = alpha * beta exactly, the
discrete counterpart of the classical sqrt(alpha*beta) result.

This module assembles and solves the voxel scheme with its own small sparse
matrices; it shares nothing with ``assembly``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _diff2d(N: int, d: int):
    S = sp.csr_matrix((np.ones(N), (np.arange(N), (np.arange(N) + 1) % N)), shape=(N, N))
    D1 = S - sp.identity(N, format="csr")
    Id = sp.identity(N, format="csr")
    return sp.kron(D1, Id, format="csr") if d == 0 else sp.kron(Id, D1, format="csr")


def ahom_voxel_2d(W: np.ndarray) -> np.ndarray:
    """2x2 homogenized matrix of the voxel scheme for the voxel field W (N,N)."""
    N = W.shape[0]
    k = [2.0 * W * np.roll(W, -1, axis=d) / (W + np.roll(W, -1, axis=d)) for d in range(2)]
    D = [_diff2d(N, d) for d in range(2)]
    A = sum(D[d].T @ sp.diags(k[d].ravel()) @ D[d] for d in range(2)).tocsc()
    # pin the constant: fix u[0] = 0 by removing row/col 0, then re-centre
    keep = np.arange(1, N * N)
    Ar = A[keep][:, keep]
    H = np.zeros((2, 2))
    for i in range(2):
        b = -(D[i].T @ k[i].ravel())
        u = np.zeros(N * N)
        u[keep] = spla.spsolve(Ar, b[keep])
        for j in range(2):
            H[i, j] = (1.0 if i == j else 0.0) * k[j].mean() + np.mean(k[j].ravel() * (D[j] @ u))
    return H
