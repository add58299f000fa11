"""Homogenized matrix of one realization (Sec. 3.4).

Test infrastructure only (see ``oracle/__init__``).

Eq. 21: Abar e_i = int a (e_i + grad phi_i). On the grid (grid units, phi_i =
h psi_i, grad phi = D psi) the j-th component of the flux is averaged over the
x_j-edges, where a_j and D_j psi_i live:

    A_ij = delta_ij * mean(a_j) + mean(a_j * D_j psi_i)          (edge form)

Summation by parts turns the second term into -(b_j . psi_i) / N^3 with
b_j = -D_j^T a_j, which is the paper's computational form (Eq. 23:
a_ii = lambda + beta <ahat> - <f_i phi_i>, a_ij = -<f_j phi_i>), since
mean(a_j) equals the volume mean of a. The symmetric energy form
mean(sum_d a_d (delta_id + D_d psi_i)(delta_jd + D_d psi_j)) agrees with both at
convergence (the paper's symmetry remark after Eq. 23).
"""
from __future__ import annotations

import numpy as np


def _fwd(psi: np.ndarray, d: int) -> np.ndarray:
    return np.roll(psi, -1, axis=d) - psi


def ahom_edge(a_edges: np.ndarray, psis) -> np.ndarray:
    """Edge form; psis[i] is the (N,N,N) corrector for e_i (any missing
    corrector may be None, its row is then left as NaN)."""
    A = np.full((3, 3), np.nan)
    for i in range(3):
        if psis[i] is None:
            continue
        for j in range(3):
            A[i, j] = (1.0 if i == j else 0.0) * a_edges[j].mean() + np.mean(a_edges[j] * _fwd(psis[i], j))
    return A


def ahom_rhs_form(a_edges: np.ndarray, bs, psis) -> np.ndarray:
    """Eq. 23 form: delta_ij mean(a) - (b_j . psi_i)/N^3."""
    A = np.full((3, 3), np.nan)
    nn = a_edges[0].size
    for i in range(3):
        if psis[i] is None:
            continue
        for j in range(3):
            A[i, j] = (1.0 if i == j else 0.0) * a_edges[j].mean() - float(np.dot(bs[j].ravel(), psis[i].ravel())) / nn
    return A


def ahom_energy(a_edges: np.ndarray, psis) -> np.ndarray:
    """Symmetric energy form; needs all three correctors."""
    g = [[(1.0 if i == d else 0.0) + _fwd(psis[i], d) for d in range(3)] for i in range(3)]
    A = np.empty((3, 3))
    for i in range(3):
        for j in range(3):
            A[i, j] = np.mean(sum(a_edges[d] * g[i][d] * g[j][d] for d in range(3)))
    return A
