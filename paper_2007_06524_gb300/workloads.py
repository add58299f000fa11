"""Named workload presets (synthetic random checkerboards).

The paper's experiments (Sec. 5) use random checkerboards generated on the
fly; no dataset exists. These presets fix the lattice, grid, contrast, seeds,
right-hand sides, preconditioner ranks, tolerance and precision of each
measured configuration. rank 0 = exact Fourier diagonal.
"""

PLAIN_N16 = dict(
    name="plain L=4 n=4 (N=16), Bernoulli(1/2) on {1,10}, seed 0, e_1, FP64, exact and R=6, tol 1e-10",
    L=4, n=4, p_hi=0.5, a_lo=1.0, a_hi=10.0, seeds=[0], dirs=[0], ranks=[0, 6], tol=1e-10, precision="fp64")

PLAIN_N256 = dict(
    name="plain L=32 n=8 (N=256), Bernoulli(1/2) on {1,100}, e_1..e_3, FP64 PCG, R in {4,8,16}, tol 1e-8",
    L=32, n=8, p_hi=0.5, a_lo=1.0, a_hi=100.0, seeds=list(range(8)), dirs=[0, 1, 2], ranks=[4, 8, 16],
    tol=1e-8, precision="fp64")

REFINE_N512 = dict(
    name="precision L=64 n=8 (N=512), Bernoulli(1/2) on {1,100}, FP32 PCG in FP64 refinement, tol 1e-10",
    L=64, n=8, p_hi=0.5, a_lo=1.0, a_hi=100.0, seeds=list(range(4)), dirs=[0, 1, 2], ranks=[0, 8],
    tol=1e-10, precision="fp32_refine", oracle_L=16)

BATCH_MIXED = dict(
    name="batching: 256 seeds x 3 RHS, L in {8,12,16,24}, n=4, Bernoulli(1/2) on {1,10}, tol 1e-8",
    Ls=[8, 12, 16, 24], n=4, p_hi=0.5, a_lo=1.0, a_hi=10.0, seeds=list(range(256)), dirs=[0, 1, 2], ranks=[0],
    tol=1e-8, precision="fp32_refine")

WARM_N64 = dict(
    name="learned warm start: L=16 n=4 (N=64), Bernoulli(1/2) on {1,10}, tol 1e-8",
    L=16, n=4, p_hi=0.5, a_lo=1.0, a_hi=10.0, train_seeds=list(range(1000, 5096)),
    eval_seeds=list(range(6000, 6512)), dirs=[0, 1, 2], ranks=[0], tol=1e-8)


def batch_L_index(seed: int) -> int:
    """Which of BATCH_MIXED['Ls'] realization `seed` uses: a seeded uniform draw."""
    import numpy as np

    return int(np.random.default_rng(seed).integers(4))
