"""Stiffness matrix and right-hand sides of the periodic corrector problem.

Test infrastructure only (see ``oracle/__init__``).

Grid (Sec. 3.1): the unit cube holds an L^3 lattice of cells, each cell has n
grid intervals per side, h = 1/(nL). The paper counts n1 = nL + 1 points per
axis with the last point identified with the first by periodicity; this
oracle stores the N = nL distinct points per axis. Node (j1, j2, j3) has the
linear index j3 + N*j2 + N^2*j1 (big-endian, x3 fastest, Sec. 3.2).

Two independent assemblies of the same matrix are provided:

* :func:`stiffness_kron_cells` follows Sec. 3.3 literally: every cell k adds
  a_k * (Qbar_k (x) Ibar_k (x) Ibar_k + Ibar_k (x) Qbar_k (x) Ibar_k
  + Ibar_k (x) Ibar_k (x) Qbar_k) (Eq. 18), with the local blocks
  Qhat = tridiag{1,-2,1} + diag{1,0,...,0,1} and Ihat = diag{1/2,1,...,1,1/2}
  of size n+1 (the n+1 grid points of the cell per axis) placed with
  periodic wrap (the "periodization" of Eqs. 12-13). Summed over all cells
  with a_k = lambda + beta*ahat_k this is lambda*A_Delta + beta*A_s (Eq. 9).
  The paper prints Qhat with the negative-semidefinite sign of the Neumann
  Laplacian (Eq. 13); this oracle uses the symmetric positive semidefinite
  stiffness, i.e. the negated block.
* :func:`stiffness_edges` writes the same operator as
  sum_d D_d^T diag(a_d) D_d with the Kronecker-structured periodic forward
  difference D_1 = (S - I) (x) I (x) I (and likewise for d = 2, 3; compare
  Eq. 14), where a_d(j) is the coefficient of the grid edge j -> j + e_d.
  Summing the Ihat weights of the cells that share an edge gives a_d(j) =
  mean of the (up to four) cells touching that edge (the nodal weights
  1, 1/2, 1/4 of Sec. 3.3, Fig. 4), i.e. the mean of the four grid voxels
  around the edge. The tests check that both assemblies agree.

Right-hand side (Eq. 8, integrated by parts, grid units): b_i = -D_i^T a_i,
i.e. b_i(j) = a_i(j) - a_i(j - e_i); sum_j b_i(j) = 0 exactly. The physical
corrector is phi_i = h * psi_i where A psi_i = b_i.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def voxel_field(cellval: np.ndarray, n: int) -> np.ndarray:
    """Coefficient of every grid voxel [v, v+1]^3 (constant per cell), shape (N,N,N)."""
    return np.repeat(np.repeat(np.repeat(cellval, n, axis=0), n, axis=1), n, axis=2)


def inclusion_field(phase: np.ndarray, n: int, sub: int, a_lo: float, a_hi: float) -> np.ndarray:
    """Voxel coefficients with sub-cell inclusions (Sec. 3.1): every unit cell
    holds a centred cube S_s of side sub grid intervals (sub = 2 alpha n); a
    voxel is a_hi when its cell is high and it lies in that cube, else a_lo
    (a = lambda + beta * indicator, lambda = a_lo). sub = n is the checkerboard."""
    if sub < 1 or sub > n or (n - sub) % 2:
        raise ValueError("sub must be in [1, n] with n - sub even (a centred cube)")
    lo = (n - sub) // 2
    u = np.arange(n)
    inside1 = (u >= lo) & (u < lo + sub)
    inside = inside1[:, None, None] & inside1[None, :, None] & inside1[None, None, :]
    hi_cell = np.repeat(np.repeat(np.repeat(phase.astype(bool), n, 0), n, 1), n, 2)
    L = phase.shape[0]
    inside_all = np.tile(inside, (L, L, L))
    return np.where(hi_cell & inside_all, float(a_hi), float(a_lo))


def level_field(level: np.ndarray, n: int, values, sub: int | None = None) -> np.ndarray:
    """Voxel coefficients of a multi-level medium (varying contrast, Sec. 2):
    cell level l carries the value values[min(l, K-1)] on its centred
    inclusion cube of side sub (Sec. 3.1; None or n = the whole cell) and
    values[0] everywhere else. K = 2 is :func:`inclusion_field`."""
    if sub is None:
        sub = n
    if sub < 1 or sub > n or (n - sub) % 2:
        raise ValueError("sub must be in [1, n] with n - sub even (a centred cube)")
    v = np.asarray(values, dtype=np.float64)
    lv = np.minimum(level.astype(np.int64), len(v) - 1)
    lo = (n - sub) // 2
    u = np.arange(n)
    inside1 = (u >= lo) & (u < lo + sub)
    inside = inside1[:, None, None] & inside1[None, :, None] & inside1[None, None, :]
    L = level.shape[0]
    cell_v = np.repeat(np.repeat(np.repeat(v[lv], n, 0), n, 1), n, 2)
    return np.where(np.tile(inside, (L, L, L)), cell_v, v[0])


def edge_coefficients(cellval: np.ndarray, n: int) -> np.ndarray:
    """a_d(j) for d = 0, 1, 2 (axes x1, x2, x3), shape (3, N, N, N), of the
    checkerboard with cell values cellval; see edge_coefficients_voxels."""
    return edge_coefficients_voxels(voxel_field(cellval, n))


def edge_coefficients_voxels(V: np.ndarray) -> np.ndarray:
    """a_d(j) for d = 0, 1, 2 (axes x1, x2, x3) of the voxel field V, shape (3, N, N, N).

    a_d(j) is the mean of the four voxels that share the edge j -> j + e_d:
    voxel index j along d, and j_t - 1 or j_t along each transverse axis t.
    np.roll(V, 1, axis=t)[j] == V[j - e_t] (periodic).
    """
    out = np.empty((3,) + V.shape)
    for d in range(3):
        t1, t2 = [t for t in range(3) if t != d]
        Vt1 = np.roll(V, 1, axis=t1)
        out[d] = 0.25 * (V + Vt1 + np.roll(V, 1, axis=t2) + np.roll(Vt1, 1, axis=t2))
    return out


def _neumann_blocks(n: int):
    """Local (n+1)x(n+1) blocks of Sec. 3.3: Qhat (negated, PSD) and Ihat."""
    m = n + 1
    Q = np.zeros((m, m))
    for i in range(m - 1):  # one unit-weight 1D edge i -> i+1
        Q[i, i] += 1.0
        Q[i + 1, i + 1] += 1.0
        Q[i, i + 1] -= 1.0
        Q[i + 1, i] -= 1.0
    Ih = np.ones(m)
    Ih[0] = Ih[-1] = 0.5
    return Q, np.diag(Ih)


def stiffness_kron_cells(cellval: np.ndarray, n: int) -> sp.csr_matrix:
    """Sum over cells of a_k times the cell's Kronecker-sum block (Eq. 18).

    Dense local block K = Q(x)I(x)I + I(x)Q(x)I + I(x)I(x)Q of size (n+1)^3,
    scattered to the cell's nodes with periodic wrap. Intended for small grids.
    """
    L = cellval.shape[0]
    N = L * n
    Q, Ih = _neumann_blocks(n)
    K = np.kron(np.kron(Q, Ih), Ih) + np.kron(np.kron(Ih, Q), Ih) + np.kron(np.kron(Ih, Ih), Q)
    kr, kc = np.nonzero(K)
    kv = K[kr, kc]
    m = n + 1
    loc = np.arange(m)
    rows, cols, vals = [], [], []
    for c1 in range(L):
        g1 = (c1 * n + loc) % N
        for c2 in range(L):
            g2 = (c2 * n + loc) % N
            for c3 in range(L):
                g3 = (c3 * n + loc) % N
                gidx = (g3[None, None, :] + N * g2[None, :, None] + N * N * g1[:, None, None]).ravel()
                rows.append(gidx[kr])
                cols.append(gidx[kc])
                vals.append(cellval[c1, c2, c3] * kv)
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N ** 3, N ** 3)
    )
    return A.tocsr()


def forward_difference(N: int, d: int) -> sp.csr_matrix:
    """Periodic forward difference along axis d: (D psi)(j) = psi(j + e_d) - psi(j)."""
    S = sp.csr_matrix((np.ones(N), (np.arange(N), (np.arange(N) + 1) % N)), shape=(N, N))
    D1 = S - sp.identity(N, format="csr")
    Id = sp.identity(N, format="csr")
    facs = [Id, Id, Id]
    facs[d] = D1
    return sp.kron(sp.kron(facs[0], facs[1]), facs[2], format="csr")


def stiffness_edges(a_edges: np.ndarray) -> sp.csr_matrix:
    """A = sum_d D_d^T diag(a_d) D_d (symmetric, A 1 = 0)."""
    N = a_edges.shape[1]
    A = None
    for d in range(3):
        D = forward_difference(N, d)
        term = D.T @ sp.diags(a_edges[d].ravel()) @ D
        A = term if A is None else A + term
    return A.tocsr()


def rhs(a_edges: np.ndarray, i: int) -> np.ndarray:
    """b_i = -D_i^T a_i (flattened), the discrete form of Eq. 8 in grid units."""
    N = a_edges.shape[1]
    D = forward_difference(N, i)
    return -(D.T @ a_edges[i].ravel())


def apply_stencil(a_edges: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Matrix-free form of A psi on an (N,N,N) field:
    sum_d a_d(j)(psi(j) - psi(j+e_d)) + a_d(j-e_d)(psi(j) - psi(j-e_d)).

    Independent of the sparse assembly; used to cross-check it.
    """
    out = np.zeros_like(psi)
    for d in range(3):
        up = np.roll(psi, -1, axis=d)      # psi(j + e_d)
        dn = np.roll(psi, 1, axis=d)       # psi(j - e_d)
        a_dn = np.roll(a_edges[d], 1, axis=d)  # a_d(j - e_d)
        out += a_edges[d] * (psi - up) + a_dn * (psi - dn)
    return out


def edge_coefficient_at(cellval: np.ndarray, n: int, d: int, j) -> float:
    """a_d(j) at one node from the definition: mean of the four voxels around
    the edge j -> j+e_d (voxel v has the value of cell v // n)."""
    L = cellval.shape[0]
    N = L * n
    t1, t2 = [t for t in range(3) if t != d]
    s = 0.0
    for s1 in (0, 1):
        for s2 in (0, 1):
            v = list(j)
            v[t1] = (j[t1] - s1) % N
            v[t2] = (j[t2] - s2) % N
            s += cellval[v[0] // n, v[1] // n, v[2] // n]
    return 0.25 * s


def apply_at(cellval: np.ndarray, n: int, psi_at, j) -> float:
    """(A psi)(j) at one node; psi_at(k) returns psi at node k (tuple)."""
    N = cellval.shape[0] * n
    out = 0.0
    pj = psi_at(tuple(j))
    for d in range(3):
        up = list(j)
        up[d] = (j[d] + 1) % N
        dn = list(j)
        dn[d] = (j[d] - 1) % N
        out += edge_coefficient_at(cellval, n, d, j) * (pj - psi_at(tuple(up)))
        out += edge_coefficient_at(cellval, n, d, tuple(dn)) * (pj - psi_at(tuple(dn)))
    return out


def rhs_at(cellval: np.ndarray, n: int, i: int, j) -> float:
    """b_i(j) = a_i(j) - a_i(j - e_i) at one node."""
    N = cellval.shape[0] * n
    dn = list(j)
    dn[i] = (j[i] - 1) % N
    return edge_coefficient_at(cellval, n, i, j) - edge_coefficient_at(cellval, n, i, tuple(dn))
