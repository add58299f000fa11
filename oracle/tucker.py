"""The paper's own rank-structured preconditioner: Tucker decomposition of
G+, Tucker-to-canonical, and the rank-(2R+1) split of Lemma 4.2.

Test infrastructure only (see ``oracle/__init__``).

Sec. 4.2 builds the canonical factors of G+ (Eqs. 32-33) in two steps: a
Tucker decomposition of the 3D tensor G+ (computed in the paper by the
multigrid Tucker algorithm of its reference KhKh3:08, which accelerates the
higher-order SVD by coarse-to-fine initial guesses), then a
Tucker-to-canonical transform of the small core. The paper states neither
algorithm. This oracle takes the plain definitions:

* Tucker (HOSVD, De Lathauwer, De Moor & Vandewalle, SIMAX 2000): the
  factor U (N x r) holds the r leading left singular vectors of the mode-1
  unfolding of G+; G+ is symmetric under any permutation of its three
  indices, so the same U serves every mode. Core beta = G+ x1 U^T x2 U^T
  x3 U^T; G_r = beta x1 U x2 U x3 U.
* Tucker-to-canonical: each mode-3 slice beta[:, :, c] of the core is a
  symmetric r x r matrix; its eigen-decomposition sum_s sigma_s e_s e_s^T
  gives the rank-1 terms sigma_s (U e_s) (x) (U e_s) (x) U[:, c]. Keeping
  every term reproduces G_r exactly (rank r^2); dropping the terms with
  |sigma_s| <= tol * max|sigma| trades accuracy for rank.
* Split (Lemma 4.2): G+ = G_1 + G_{n-1} with G_1 the k1 = 0 slice of G+ and
  G_{n-1} the rest. With an exponential sum sum_r w_r exp(-t_r x) for 1/x
  (Eq. 34), G_{n-1} has the R terms w_r ([k != 0] e_r) (x) e_r (x) e_r,
  e_r(k) = exp(-t_r lambda_k), and G_1 the R terms w_r delta_0 (x) e_r (x) e_r
  plus one term -(sum_r w_r) delta_0 (x) delta_0 (x) delta_0 that clears the
  (0, 0, 0) entry: 2R + 1 terms in all.

Pinned by: exact reproduction at full rank, the HOSVD error bounds
(between the discarded singular values of one mode and three times their
sum of squares), exact Tucker-to-canonical at tol = 0, evenness of the
factors, and the identity of the split with the exponential-sum tensor whose
zero mode is set to 0.
"""
from __future__ import annotations

import numpy as np

from . import precond


def hosvd(G: np.ndarray, r: int):
    """(U, sigma): r leading left singular vectors of the mode-1 unfolding
    (N x N^2) of the symmetric tensor G, and all its singular values."""
    N = G.shape[0]
    U, s, _ = np.linalg.svd(G.reshape(N, N * N), full_matrices=False)
    return U[:, :r], s


def tucker_core(G: np.ndarray, U: np.ndarray) -> np.ndarray:
    """beta = G x1 U^T x2 U^T x3 U^T."""
    return np.einsum("ijk,ia,jb,kc->abc", G, U, U, U, optimize=True)


def tucker_full(U: np.ndarray, core: np.ndarray) -> np.ndarray:
    """beta x1 U x2 U x3 U."""
    return np.einsum("abc,ia,jb,kc->ijk", core, U, U, U, optimize=True)


def tucker_to_canonical(U: np.ndarray, core: np.ndarray, tol: float = 0.0):
    """Canonical factors (F1, F2, F3), each (R, N), with the weights folded
    into F1: G ~ sum_r F1[r] (x) F2[r] (x) F3[r]."""
    r = core.shape[0]
    eig = []
    for c in range(r):
        S = 0.5 * (core[:, :, c] + core[:, :, c].T)
        eig.append(np.linalg.eigh(S))
    smax = max(float(np.abs(w).max()) for w, _ in eig)
    F1, F2, F3 = [], [], []
    for c, (w, V) in enumerate(eig):
        for s in range(r):
            if abs(w[s]) > tol * smax or tol == 0.0:
                v = U @ V[:, s]
                F1.append(w[s] * v)
                F2.append(v)
                F3.append(U[:, c])
    return np.array(F1), np.array(F2), np.array(F3)


def canonical_full(F1: np.ndarray, F2: np.ndarray, F3: np.ndarray) -> np.ndarray:
    """sum_r F1[r] (x) F2[r] (x) F3[r]."""
    return np.einsum("ri,rj,rk->ijk", F1, F2, F3, optimize=True)


def lemma_split(N: int, t, w):
    """The 2R + 1 canonical factors of Lemma 4.2 for the exponential sum
    (t, w); returns (F1, F2, F3), each (2R + 1, N)."""
    lam = precond.laplacian_eigenvalues(N)
    t = np.asarray(t, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    E = np.exp(-np.outer(t, lam))  # e_r(k)
    d0 = np.zeros(N)
    d0[0] = 1.0
    nz = np.ones(N)
    nz[0] = 0.0
    F1 = np.vstack([w[:, None] * E * nz, w[:, None] * d0, [-w.sum() * d0]])
    F2 = np.vstack([E, E, [d0]])
    F3 = np.vstack([E, E, [d0]])
    return F1, F2, F3


def max_relative_error_full(N: int, G: np.ndarray) -> float:
    """max over nonzero modes of |g G(k) - 1|, g = l1 + l2 + l3."""
    lam = precond.laplacian_eigenvalues(N)
    g = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    nz = g > 0
    return float(np.abs(g[nz] * G[nz] - 1.0).max())
