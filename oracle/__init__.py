"""CPU oracle for the periodic corrector problem on a random checkerboard.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The GPU product path (``paper_2007_06524_gb300``) never imports it and
shares no code, table or constant generator with it.

Everything here is plain FP64 numpy / scipy, written to be checked against the
paper (Khoromskaia & Khoromskij, "Tensor-based techniques for fast
discretization and solution of 3D elliptic equations with random
coefficients", arXiv 2007.06524) by eye:

* ``rng``          -- SplitMix64 counter stream and the checkerboard cell phases
                      (coefficient model, Sec. 2, Eq. 3).
* ``assembly``     -- stiffness matrix as the paper's Kronecker sum over cells
                      (Sec. 3.3, Eqs. 16-18) and as the equivalent edge form
                      sum_d D_d^T diag(a_d) D_d; right-hand sides (Eq. 8).
* ``precond``      -- Laplacian eigenvalues (Eqs. 28-29), the pseudo-inverse
                      core tensor G^+ (Eqs. 32-33), its rank-R canonical
                      approximation (Eq. 34, Lemma 4.2) and the FFT apply
                      (Eq. 31).
* ``tucker``       -- the paper's Tucker route to the canonical factors
                      (HOSVD of G^+, Tucker-to-canonical, Sec. 4.2) and the
                      2R+1 split of Lemma 4.2.
* ``pcg``          -- CG / PCG on the zero-mean subspace (Eqs. 24-25) and the
                      tight / dense reference solves.
* ``homogenized``  -- the homogenized matrix (Eqs. 21-23).
* ``solver2d``     -- the 2D corrector problem of the paper's 2D experiments
                      (node scheme, 2D preconditioner, PCG, 2 x 2 A_hom).
* ``dual2d``       -- an independent 2D cell-centred scheme used only to pin the
                      node scheme through discrete Keller duality.

Parity status of each function is stated in its docstring. The rank-R
node placements (trapezoid rule, and geometric nodes with least-squares
weights) are readings of ours (the paper gives none); both are pinned by
their convergence to the exact G+ as R grows, the least-squares fit also by
its normal equations and by beating the trapezoid rule, and the Tucker route
by the HOSVD error bounds (tests/test_oracle_*).
"""
