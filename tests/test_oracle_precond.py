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


# ----------------------------------------------- least-squares exponential sum
@pytest.mark.parametrize("N,dim", [(6, 3), (8, 3), (12, 3), (8, 2), (18, 2)])
def test_spectrum_values_brute_force(N, dim):
    """The distinct nonzero eigenvalues from the half index range equal the
    distinct values of the full Kronecker-sum spectrum (brute force over all
    N^dim index tuples, deduplicated by rounding)."""
    lam = precond.laplacian_eigenvalues(N)
    full = lam[:, None] + lam[None, :] if dim == 2 else lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    ref = np.unique(np.round(full.ravel(), 10))
    ref = ref[ref > 0]
    got = precond.spectrum_values(N, dim)
    assert len(got) == len(ref) and np.allclose(got, ref, rtol=0, atol=1e-9)


def test_log_uniform_sample_members():
    v = precond.spectrum_values(64)
    x = precond.log_uniform_sample(v)
    assert x[0] == v[0] and x[-1] == v[-1]
    assert np.all(np.diff(x) > 0) and np.all(np.isin(x, v))
    # nearest value to each point of a geometric grid of 3000 points: a value
    # farther than two grid steps (in log x) from both neighbours is always
    # picked
    step = np.log(v[-1] / v[0]) / 2999
    lv = np.log(v)
    gap = np.minimum(np.diff(lv, prepend=-np.inf), -np.diff(lv, append=np.inf))
    assert np.all(np.isin(v[gap > 2 * step], x))
    assert len(x) <= 3000


@pytest.mark.parametrize("N,R,dim", [(16, 6, 3), (64, 8, 3), (256, 8, 3), (64, 16, 3), (256, 8, 2), (48, 4, 3),
                                     (16, 16, 3), (24, 32, 3)])
def test_lsq_sum_positive_geometric_and_better_than_trapezoid(N, R, dim):
    t, w = precond.lsq_nodes(N, R, dim)
    assert np.all(t > 0) and np.all(w > 0)
    assert np.allclose(t[1:] / t[:-1], t[1] / t[0], rtol=1e-12)      # geometric nodes
    v = precond.spectrum_values(N, dim)
    e_fit = precond.sampled_relative_error(v, t, w)
    e_trap = precond.sampled_relative_error(v, *precond.rank_r_nodes(N, R, dim))
    assert e_fit <= e_trap


@pytest.mark.parametrize("N,R", [(64, 8), (256, 8), (32, 16)])
def test_lsq_weights_satisfy_normal_equations(N, R):
    """Least squares (textbook): at the fitted weights the residual of
    min ||E w - 1|| on the sample is orthogonal to the columns of E, and any
    other weights on the same nodes (e.g. the trapezoid weights rescaled)
    give a larger residual."""
    t, w = precond.lsq_nodes(N, R)
    x = precond.log_uniform_sample(precond.spectrum_values(N))
    E = x[:, None] * np.exp(-np.outer(x, t))
    res = E @ w - 1.0
    assert np.abs(E.T @ res).max() <= 1e-9 * np.linalg.norm(E, axis=0).max() * max(np.linalg.norm(res), 1e-300) * 1e3
    rng_ = np.random.default_rng(0)
    for _ in range(5):
        dw = rng_.standard_normal(R) * 1e-3 * w
        assert np.linalg.norm(E @ (w + dw) - 1.0) >= np.linalg.norm(res)


@pytest.mark.parametrize("N", [32, 64, 256])
def test_lsq_sum_converges_to_exact(N):
    """More terms, smaller error: the fit approaches G+ = 1/x (Eq. 33)."""
    v = precond.spectrum_values(N)
    errs = [precond.sampled_relative_error(v, *precond.lsq_nodes(N, R)) for R in (4, 8, 16)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3


def test_lsq_above_32_terms_is_the_trapezoid_rule():
    t, w = precond.lsq_nodes(16, 40)
    ts, ws = precond.rank_r_nodes(16, 40)
    assert np.array_equal(t, ts) and np.array_equal(w, ws)
