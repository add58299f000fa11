"""The 2D corrector problem (Sec. 5, the 2D experiments): node scheme,
right-hand sides, the 2D spectral preconditioner, PCG and the 2 x 2 A_hom.

Test infrastructure only (see ``oracle/__init__``).

The paper's 2D study (n0 grid intervals per cell, L^2 cells, overlap factor
alpha) solves -div(a(e_i + grad phi_i)) = 0, i = 1, 2, on the periodic unit
square with the same construction as in 3D, one dimension down:

* Cells: the L x L lattice, cell (c1, c2) high iff the top 53 bits of
  SplitMix64 output number c2 + L c1 are below floor(p_hi 2^53) -- the 3D
  rule on the slab c1 = 0 (``rng``), so a 2D realization is the first x1-slab
  of the 3D one with the same L and seed. Sub-cell inclusions as in 3D: a
  centred square of side sub grid intervals per cell.
* Node scheme (Sec. 3 in 2D): grid N = L n per axis, node (j1, j2), voxel
  v = [v1, v1+1] x [v2, v2+1]. The lumped Q1 edge coefficient a_d(j) of the
  edge j -> j + e_d is the mean of the two voxels beside it: voxel index j_d
  along d and j_t - 1 or j_t along the other axis t.
  A = sum_d D_d^T diag(a_d) D_d with periodic forward differences D_d;
  b_i = -D_i^T a_i.
* Preconditioner (Sec. 4 in 2D): G(k1, k2) = 1 / (lambda_k1 + lambda_k2),
  G(0, 0) = 0, applied with the 2D FFT; its rank-R form is the exponential
  sum sum_r w_r exp(-t_r (lambda_k1 + lambda_k2)).
* A_hom (Eq. 21 in 2D): A_ij = delta_ij mean(a_j) + mean(a_j D_j psi_i); the
  energy form beside it.

Pinned by: the x3-invariant 3D oracle (its 2 x 2 block equals this scheme),
Keller's duality against the independent voxel scheme of ``dual2d``, the
checkerboard product alpha beta, the laminate closed form, the Fourier
eigenvalues of the constant-coefficient operator, and a manufactured
solution.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import pcg as _pcg
from . import precond, rng


def cell_phases_2d(L: int, seed: int, p_hi: float = 0.5) -> np.ndarray:
    """Phase of every cell (L, L): the 3D draw's slab c1 = 0."""
    thr = rng.hi_threshold(p_hi)
    ph = np.zeros((L, L), dtype=np.uint8)
    for c1 in range(L):
        for c2 in range(L):
            ph[c1, c2] = 1 if (rng.splitmix64_at(seed, c2 + L * c1) >> 11) < thr else 0
    return ph


def cell_phases_2d_vec(L: int, seed: int, p_hi: float = 0.5) -> np.ndarray:
    """Same as :func:`cell_phases_2d`, vectorised with numpy uint64 (checked
    against it in the tests); used for large L."""
    thr = np.uint64(rng.hi_threshold(p_hi))
    idx = np.arange(L * L, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & rng.MASK64) + (idx + np.uint64(1)) * np.uint64(rng.GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(rng.MIX_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(rng.MIX_M2)
        z = z ^ (z >> np.uint64(31))
    return ((z >> np.uint64(11)) < thr).astype(np.uint8).reshape(L, L)


def voxel_field_2d(phase: np.ndarray, n: int, a_lo: float, a_hi: float, sub: int | None = None) -> np.ndarray:
    """Voxel coefficients (N, N): a_hi where the cell is high and the voxel lies
    in the cell's centred square of side sub (None = the whole cell), else a_lo."""
    if sub is None:
        sub = n
    if sub < 1 or sub > n or (n - sub) % 2:
        raise ValueError("sub must be in [1, n] with n - sub even")
    lo = (n - sub) // 2
    u = np.arange(n)
    in1 = (u >= lo) & (u < lo + sub)
    inside = np.tile(in1[:, None] & in1[None, :], phase.shape)
    hi = np.repeat(np.repeat(phase.astype(bool), n, 0), n, 1)
    return np.where(hi & inside, float(a_hi), float(a_lo))


def edge_coefficients_2d(V: np.ndarray) -> np.ndarray:
    """a_d(j), d = 0, 1, shape (2, N, N): mean of the two voxels beside the edge
    j -> j + e_d (np.roll(V, 1, axis=t)[j] = V[j - e_t])."""
    out = np.empty((2,) + V.shape)
    for d in range(2):
        t = 1 - d
        out[d] = 0.5 * (V + np.roll(V, 1, axis=t))
    return out


def _diff(N: int, d: int) -> sp.csr_matrix:
    S = sp.csr_matrix((np.ones(N), (np.arange(N), (np.arange(N) + 1) % N)), shape=(N, N))
    D1 = S - sp.identity(N, format="csr")
    Id = sp.identity(N, format="csr")
    return sp.kron(D1, Id, format="csr") if d == 0 else sp.kron(Id, D1, format="csr")


def stiffness_2d(a: np.ndarray) -> sp.csr_matrix:
    N = a.shape[1]
    D = [_diff(N, d) for d in range(2)]
    return sum(D[d].T @ sp.diags(a[d].ravel()) @ D[d] for d in range(2)).tocsr()


def rhs_2d(a: np.ndarray, i: int) -> np.ndarray:
    """b_i = -D_i^T a_i, i.e. b_i(j) = a_i(j) - a_i(j - e_i)."""
    return (a[i] - np.roll(a[i], 1, axis=i)).ravel()


def core_2d_exact(N: int) -> np.ndarray:
    lam = precond.laplacian_eigenvalues_fft(N)
    g = lam[:, None] + lam[None, :]
    G = np.zeros_like(g)
    G[g > 0] = 1.0 / g[g > 0]
    return G


def core_2d_from_nodes(N: int, t, w) -> np.ndarray:
    """sum_r w_r exp(-t_r (l1 + l2)), G(0, 0) := 0."""
    lam = precond.laplacian_eigenvalues(N)
    g = lam[:, None] + lam[None, :]
    G = np.exp(-np.multiply.outer(g, np.asarray(t, dtype=np.float64))) @ np.asarray(w, dtype=np.float64)
    G[0, 0] = 0.0
    return G


def apply_precond_2d(G: np.ndarray, r: np.ndarray) -> np.ndarray:
    return np.real(np.fft.ifft2(G * np.fft.fft2(r)))


def ahom_2d(a: np.ndarray, psis) -> np.ndarray:
    """Edge form, 2 x 2."""
    H = np.zeros((2, 2))
    for i in range(2):
        for j in range(2):
            H[i, j] = (1.0 if i == j else 0.0) * a[j].mean() + np.mean(a[j] * (np.roll(psis[i], -1, axis=j) - psis[i]))
    return H


def ahom_2d_energy(a: np.ndarray, psis) -> np.ndarray:
    H = np.zeros((2, 2))
    g = [[(1.0 if i == d else 0.0) + np.roll(psis[i], -1, axis=d) - psis[i] for d in range(2)] for i in range(2)]
    for i in range(2):
        for j in range(2):
            H[i, j] = np.mean(sum(a[d] * g[i][d] * g[j][d] for d in range(2)))
    return H


def solve_2d(V: np.ndarray, tol: float = 1e-13, G=None):
    """Both correctors of the voxel field V by PCG with the 2D preconditioner
    (G: core tensor, default exact); returns (psis, iterations, A_hom, a)."""
    N = V.shape[0]
    a = edge_coefficients_2d(V)
    A = stiffness_2d(a)
    G = core_2d_exact(N) if G is None else G
    P = lambda r: apply_precond_2d(G, r.reshape(N, N)).ravel()
    psis, its = [], []
    for i in range(2):
        x, it, _ = _pcg.pcg(A, rhs_2d(a, i), P, tol=tol, maxit=20000)
        psis.append(x.reshape(N, N))
        its.append(it)
    return psis, its, ahom_2d(a, psis), a
