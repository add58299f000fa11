"""Pins for the oracle's preconditioner (Sec. 4.2)."""
import numpy as np
import pytest

from oracle import assembly, pcg, precond


@pytest.mark.parametrize("N", [4, 7, 16, 48, 256])
def test_eigenvalues_fft_closed_form(N):
    assert np.allclose(precond.laplacian_eigenvalues_fft(N), precond.laplacian_eigenvalues(N), atol=1e-13)


@pytest.mark.parametrize("N", [5, 8, 12])
def test_eigenvalues_match_dense_circulant(N):
    # library eigen-solver on the explicit periodic 1D Laplacian
    P = 2 * np.eye(N) - np.roll(np.eye(N), 1, axis=1) - np.roll(np.eye(N), -1, axis=1)
    assert np.allclose(np.sort(np.linalg.eigvalsh(P)), np.sort(precond.laplacian_eigenvalues(N)), atol=1e-12)


def test_exact_precond_is_laplacian_pseudoinverse():
    N = 4
    A_lap = assembly.stiffness_edges(assembly.edge_coefficients(np.ones((2, 2, 2)), 2)).toarray()
    Pinv = np.linalg.pinv(A_lap)
    r = np.random.default_rng(1).standard_normal((N, N, N))
    z = precond.apply_precond(precond.core_tensor_exact(N), r)
    assert np.allclose(z.ravel(), Pinv @ r.ravel(), atol=1e-12)
    assert abs(z.mean()) < 1e-14


def test_exact_pcg_one_iteration_on_constant_coefficient():
    # a = c: A = c A_Delta and P = A_Delta^+, so P A = I/c on <u,1> = 0
    N, c = 8, 2.5
    a = assembly.edge_coefficients(np.full((4, 4, 4), c), 2)
    A = assembly.stiffness_edges(a)
    f = np.random.default_rng(2).standard_normal(N ** 3)
    f -= f.mean()
    x, it, rel = pcg.pcg(A, f, pcg.fft_preconditioner(N, 0), tol=1e-12)
    assert it == 1 and rel < 1e-12


@pytest.mark.parametrize("N", [16, 32])
def test_rank_r_weights_positive_and_converging(N):
    E = precond.core_tensor_exact(N)
    m = E > 0
    errs = []
    for R in (4, 8, 16, 32, 64):
        t, w = precond.rank_r_nodes(N, R)
        assert np.all(w > 0) and np.all(t > 0)
        G = precond.core_tensor_rank_r(N, R)
        assert G[0, 0, 0] == 0.0 and np.all(G[m] > 0)
        errs.append(np.abs(G[m] / E[m] - 1).max())
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    assert errs[-1] < 1e-7          # the quadrature reaches the exact G+ (Eq. 33)


def test_rank_r_symmetric_factorisation():
    N, R = 12, 6
    U = precond.rank_r_factors(N, R)
    G = precond.core_tensor_rank_r(N, R)
    # G_R(k1,k2,k3) is symmetric under axis permutations and even in each k
    assert np.allclose(G, G.transpose(1, 0, 2)) and np.allclose(G, G.transpose(2, 1, 0))
    k = (-np.arange(N)) % N
    assert np.allclose(G, G[k][:, k][:, :, k])
    assert np.allclose(G[1, 2, 3], np.sum(U[:, 1] * U[:, 2] * U[:, 3]))


def test_spectral_ratio_bounds():
    assert precond.spectral_ratio(32, 8) < 1.2
    assert precond.spectral_ratio(32, 16) < 1.01


def test_core_tensor_from_nodes_consistent():
    N, R = 16, 6
    t, w = precond.rank_r_nodes(N, R)
    assert np.allclose(precond.core_tensor_from_nodes(N, t, w), precond.core_tensor_rank_r(N, R), rtol=1e-14, atol=0)
    E = precond.core_tensor_exact(N)
    G = precond.core_tensor_rank_r(N, R)
    m = E > 0
    assert abs(precond.max_relative_error(N, t, w) - np.abs(G[m] / E[m] - 1).max()) < 1e-12


@pytest.mark.parametrize("L,n,sub,lo", [(2, 4, None, 0.25), (4, 2, None, 0.1), (3, 4, 2, 0.4), (4, 3, None, 0.02)])
def test_spectral_equivalence_interval(L, n, sub, lo):
    """Lemma 4.1 in its sharp form: x'Ax = sum_e a_e (Dx)_e^2 and the exact
    preconditioner is the pseudo-inverse of B with x'Bx = sum_e (Dx)_e^2, so
    every nonzero eigenvalue of P A lies in [min a_e, max a_e] (hence
    cond <= 1 / lambda for a in [lambda, 1]). The rank-8 tensor G_R is
    diagonal in the same Fourier basis as B+, with g G_R in [1 - e, 1 + e]
    (e its relative error), so its interval is [min a_e (1 - e),
    max a_e (1 + e)]."""
    from oracle import problem

    re = problem.realization(L, n, 7, lo, 1.0, 0.5, sub=sub)
    N = re.N
    a = re.a_edges
    A = re.A.toarray()
    for rank in (0, 8):
        G = precond.core_tensor(N, rank)
        PA = np.stack([precond.apply_precond(G, A[:, j].reshape(N, N, N)).ravel() for j in range(N ** 3)], axis=1)
        ev = np.linalg.eigvals(PA)
        assert np.abs(ev.imag).max() <= 1e-9  # similar to a symmetric matrix
        ev = np.sort(ev.real)
        assert np.abs(ev[0]) <= 1e-10  # the constants
        nz = ev[1:]
        e = 0.0 if rank == 0 else precond.max_relative_error(N, *precond.rank_r_nodes(N, rank))
        assert nz.min() >= a.min() * (1 - e) - 1e-10
        assert nz.max() <= a.max() * (1 + e) + 1e-10
