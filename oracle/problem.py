"""One realization of the corrector problem, end to end on the CPU.

Test infrastructure only (see ``oracle/__init__``).

realization(...) -> cells, edge coefficients, stiffness matrix, right-hand
sides; solve_correctors(...) -> the three zero-mean correctors and A_hom.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import assembly, homogenized, pcg, precond, rng


@dataclass
class Realization:
    L: int
    n: int
    N: int
    phase: np.ndarray      # (L,L,L) uint8
    cellval: np.ndarray    # (L,L,L) float64
    a_edges: np.ndarray    # (3,N,N,N) float64
    A: object              # scipy CSR, N^3 x N^3
    b: list                # three flat RHS vectors


def realization(L: int, n: int, seed: int, a_lo: float, a_hi: float, p_hi: float = 0.5,
                phase: np.ndarray | None = None, sub: int | None = None) -> Realization:
    """sub: side of the centred inclusion cube per cell in grid intervals
    (sub-cell inclusions, Sec. 3.1); None or n = the full-cell checkerboard."""
    if phase is None:
        phase = rng.cell_phases_vec(L, seed, p_hi) if L > 16 else rng.cell_phases(L, seed, p_hi)
    cellval = rng.cell_values(phase, a_lo, a_hi)
    if sub is None or sub == n:
        a_edges = assembly.edge_coefficients(cellval, n)
    else:
        a_edges = assembly.edge_coefficients_voxels(assembly.inclusion_field(phase, n, sub, a_lo, a_hi))
    A = assembly.stiffness_edges(a_edges)
    b = [assembly.rhs(a_edges, i) for i in range(3)]
    return Realization(L, n, L * n, phase, cellval, a_edges, A, b)


def realization_levels(L: int, n: int, seed: int, values, probs=None, level: np.ndarray | None = None,
                       sub: int | None = None) -> Realization:
    """Multi-level realization (varying contrast, Sec. 2): cell levels drawn
    with probabilities probs (rng.cell_levels) or given as `level`; voxel
    values from assembly.level_field. `phase` holds the levels and `cellval`
    the cell values."""
    if level is None:
        level = rng.cell_levels_vec(L, seed, probs) if L > 16 else rng.cell_levels(L, seed, probs)
    cellval = rng.level_values(level, values)
    a_edges = assembly.edge_coefficients_voxels(assembly.level_field(level, n, values, sub))
    A = assembly.stiffness_edges(a_edges)
    b = [assembly.rhs(a_edges, i) for i in range(3)]
    return Realization(L, n, L * n, level, cellval, a_edges, A, b)


def solve_correctors(re: Realization, dirs=(0, 1, 2), rank: int = 0, tol: float = 1e-13):
    """PCG-solve A psi_i = b_i for the requested directions; returns
    (psis list (None where not solved), iterations list, A_hom)."""
    P = pcg.fft_preconditioner(re.N, rank)
    psis, its = [None, None, None], [None, None, None]
    for i in dirs:
        x, it, _ = pcg.pcg(re.A, re.b[i], P, tol=tol, maxit=5000)
        psis[i] = x.reshape(re.N, re.N, re.N)
        its[i] = it
    return psis, its, homogenized.ahom_edge(re.a_edges, psis)


__all__ = ["Realization", "realization", "realization_levels", "solve_correctors", "precond"]
