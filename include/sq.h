/*
 * sq.h -- C ABI of libsq, a single-GPU (GB300, sm_103a) solver for the periodic
 * corrector problem of Khoromskaia & Khoromskij, "Tensor-based techniques for
 * fast discretization and solution of 3D elliptic equations with random
 * coefficients" (arXiv 2007.06524).
 *
 * Problem (Sec. 2, Eqs. 3-4; Sec. 3.4, Eqs. 20-21): on the unit cube with an
 * L x L x L checkerboard of cells, each cell holding a_lo or a_hi, find for
 * i = 1..3 the periodic corrector with -div(a (e_i + grad phi_i)) = 0 and
 * the homogenized matrix A_hom e_i = mean(a (e_i + grad phi_i)).
 *
 * Discretization (Sec. 3.1-3.3): N = L*n grid points per axis (n points per
 * cell side; the paper's n1 = N + 1 with the last point identified with the
 * first), node (j1,j2,j3) stored at j3 + N*j2 + N*N*j1 (x3 fastest, the
 * paper's big-endian order). The stiffness matrix is A = sum_d D_d^T
 * diag(a_d) D_d with the periodic forward difference D_d and the edge
 * coefficient a_d(j) = mean of the cells touching the edge j -> j+e_d (the
 * nodal weights 1, 1/2, 1/4 of Sec. 3.3, Eq. 18). It is never stored:
 * every kernel rebuilds the edge coefficients from the L^3 cell phases.
 * Right-hand side (Eq. 8): b_i = -D_i^T a_i. All fields are in grid units:
 * the library returns psi_i with A psi_i = b_i; the physical corrector is
 * phi_i = h * psi_i, h = 1/N.
 *
 * Conventions for every call:
 *  - Return value: SQ_OK (0) or an error code below; sq_strerror() names it.
 *  - Field pointers (double* / float*) are DEVICE pointers to N^3 contiguous
 *    elements in the layout above, owned by the caller; they must not alias
 *    each other unless stated.
 *  - Handles (sq_coeffs, sq_precond, sq_workspace) are opaque, owned by the
 *    library, created by the *_create/build/setup call and released with the
 *    matching *_destroy (NULL is accepted by destroy).
 *  - Calls are asynchronous on the given stream (a cudaStream_t; NULL = the
 *    legacy default stream) unless marked "synchronizes".
 *  - On error nothing is guaranteed about the output buffers; a CUDA error
 *    that was raised by an earlier asynchronous call may surface as SQ_ECUDA.
 *  - Handles carry reduction scratch. Calls that reduce through one
 *    sq_coeffs (sq_homogenized_matrix, sq_apply_operator[_f32], sq_rhs), and
 *    all calls on one sq_workspace, must be ordered on one stream. Solves only
 *    read their sq_coeffs and sq_precond, so the three correctors of a
 *    realization may run concurrently on separate workspaces and streams.
 *  - Options and tile choices (sq_set_option, sq_set_tiles) are process-wide
 *    and must not change while a solve runs.
 */
#ifndef SQ_H
#define SQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sq_stream_t; /* same type as cudaStream_t */

enum sq_status {
  SQ_OK = 0,
  SQ_EINVAL = 1,     /* bad argument (size, NULL, mismatched handles)          */
  SQ_ENOMEM = 2,     /* device or host allocation failed                        */
  SQ_ECUDA = 3,      /* CUDA runtime error                                      */
  SQ_ENOCONV = 4,    /* max_iter reached before the tolerance (result is valid) */
  SQ_ETIMEOUT = 5,   /* a bounded device wait gave up                           */
  SQ_EBADGUESS = 6   /* initial guess rejected, solve restarted from zero       */
};

enum sq_precision {
  SQ_FP64 = 0,        /* every field, matvec, FFT and reduction in FP64          */
  SQ_FP32_REFINE = 1  /* FP32 PCG inner solves inside FP64 iterative refinement:
                         FP64 residual, solution, norms and mean projection     */
};

typedef struct sq_coeffs sq_coeffs;
typedef struct sq_precond sq_precond;
typedef struct sq_workspace sq_workspace;

typedef struct sq_solve_info {
  int iters;          /* PCG iterations (x updates); summed over inner solves   */
  int outer_steps;    /* refinement steps (1 for SQ_FP64)                       */
  int status;         /* SQ_OK, SQ_ENOCONV or SQ_ETIMEOUT (the call's return)   */
  int used_guess;     /* 1 if x0 was used                                        */
  double relres;      /* last recurrence residual ||r||/||b||                    */
  double relres_true; /* ||b - A psi||/||b||, recomputed in FP64 after the solve */
} sq_solve_info;

/* Coefficient generation (Sec. 2, Eq. 3: a = lambda + beta*ahat per cell).
 * Cell (c1,c2,c3) is high (a_hi) iff the top 53 bits of output number
 * c3 + L*c2 + L*L*c1 of the SplitMix64 stream seeded with `seed` (Steele, Lea
 * & Flood, OOPSLA 2014), read as an integer, are below floor(p_hi * 2^53).
 * L >= 1, n >= 2, 8 <= L*n <= 512, L*n even, L*n = 2^a 3^b with b <= 1,
 * 0 <= p_hi <= 1, 0 < a_lo, 0 < a_hi. The cell phases (L^3 bytes) stay on the
 * device inside the handle. */
int sq_build_coeffs(int L, int n, uint64_t seed, double p_hi, double a_lo, double a_hi,
                    sq_stream_t stream, sq_coeffs **out);

/* Same, with the L^3 phases (0 = a_lo, nonzero = a_hi, index c3 + L*c2 + L*L*c1)
 * given in HOST memory; they are copied to the device on `stream`
 * (host_phase may be reused once the call returns: the copy is staged).
 * Nonzero bytes are stored as 1. */
int sq_coeffs_from_host(int L, int n, const uint8_t *host_phase, double a_lo, double a_hi,
                        sq_stream_t stream, sq_coeffs **out);

/* Redraws the phases of an existing handle in place from (seed, p_hi), with
 * the rule of sq_build_coeffs (no allocation; asynchronous on `stream`). */
int sq_coeffs_regenerate(sq_coeffs *c, uint64_t seed, double p_hi, sq_stream_t stream);

/* Copies L^3 phases from PINNED host memory into an existing handle
 * (cudaMemcpyAsync on `stream`: host_phase must stay valid until the stream
 * reaches the copy; values 0 or 1, or the cell levels of a multi-level
 * handle, at most 3). */
int sq_coeffs_upload(sq_coeffs *c, const uint8_t *host_phase, sq_stream_t stream);

/* Copies the phases to host_phase (L^3 bytes, may be NULL) and counts the high
 * cells into *n_hi (may be NULL). Synchronizes the handle's stream. */
int sq_coeffs_cells(const sq_coeffs *c, uint8_t *host_phase, int64_t *n_hi);
/* Grid parameters of a handle (any output may be NULL). */
int sq_coeffs_shape(const sq_coeffs *c, int *L, int *n, int *N);
/* Sub-cell inclusions (Sec. 3.1): every unit cell holds a centred cube of
 * side `sub` grid intervals (sub = 2 alpha n, alpha the paper's overlap
 * factor); a voxel takes a_hi only if its cell is high and it lies in that
 * cube, a_lo everywhere else. sub = n (the default) is the full-cell
 * checkerboard. Requires 1 <= sub <= n with n - sub even; SQ_EINVAL otherwise.
 * Applies to every later use of c (solves, batches created afterwards,
 * A_hom, the warm-start features). */
int sq_coeffs_set_subcell(sq_coeffs *c, int sub);

/* Multi-level media (varying contrast, Sec. 2: inclusion cells carry
 * lambda + beta_c with a contrast beta_c that differs between cells, drawn
 * at random or set per layer of cells). A cell's phase byte v selects level
 * min(v, K - 1) with coefficient values[level]; voxels outside the cell's
 * inclusion cube (sq_coeffs_set_subcell) take values[0]. The lumped edge
 * coefficient stays the mean of the four voxels around the edge.
 * sq_coeffs_set_levels: 2 <= K <= 4 values, each finite and > 0 (HOST
 * array, read during the call); K = 2 is the two-level medium
 * {a_lo, a_hi} = {values[0], values[1]}. Applies to every later use of c,
 * as sq_coeffs_set_subcell does. SQ_EINVAL on a bad argument. */
int sq_coeffs_set_levels(sq_coeffs *c, int K, const double *values);

/* A new K-level handle with cell levels drawn from the SplitMix64 stream of
 * sq_build_coeffs: with the top 53 bits u of the cell's output and the tail
 * probabilities P_m = probs[m] + ... + probs[K-1] (summed in FP64 from the
 * top level down), the level is the number of m in 1..K-1 with
 * u < floor(min(P_m, 1) * 2^53). K = 2 with probs = {1 - p_hi, p_hi} draws
 * the same cells as sq_build_coeffs. probs: K HOST values in [0, 1] summing
 * to 1 (within 1e-9); values as for sq_coeffs_set_levels. */
int sq_build_coeffs_levels(int L, int n, uint64_t seed, int K, const double *probs, const double *values,
                           sq_stream_t stream, sq_coeffs **out);
/* A new K-level handle with the L^3 cell levels given in HOST memory (index
 * as in sq_coeffs_from_host; bytes >= K are stored as K - 1; the copy is
 * staged, host_level may be reused once the call returns). */
int sq_coeffs_from_host_levels(int L, int n, const uint8_t *host_level, int K, const double *values,
                               sq_stream_t stream, sq_coeffs **out);
/* Redraws the levels of a K-level handle in place (K must equal the
 * handle's level count; asynchronous on `stream`, no allocation). */
int sq_coeffs_regenerate_levels(sq_coeffs *c, uint64_t seed, int K, const double *probs, sq_stream_t stream);
void sq_coeffs_destroy(sq_coeffs *c);

/* Preconditioner (Sec. 4.1-4.2): pseudo-inverse of the periodic Laplacian,
 * z = F^-1 G F r with G(k) = 1/(l_k1 + l_k2 + l_k3), l_k = 4 sin^2(pi k/N),
 * G(0,0,0) = 0 (Eqs. 31-33). rank = 0 uses this exact Fourier diagonal; rank
 * R >= 2 uses the rank-R canonical tensor G_R = sum_r u_r (x) u_r (x) u_r with
 * u_r(k) = w_r^(1/3) exp(-t_r l_k) (Lemma 4.2; the exponential sum
 * sum_r w_r exp(-t_r x) ~ 1/x of the Laplace transform, Eq. 34), R <= 64. For
 * R <= 32 the nodes are geometric and the weights fitted by least squares to
 * the relative error over the discrete spectrum (a fit counts only if it keeps
 * every weight positive and is not numerically singular: the triangular
 * factor of its QR decomposition has a diagonal spread of at most 1e10); the
 * balanced trapezoid rule is used above R = 32 and wherever no fit beats it.
 * Factors and twiddles are built on the host in FP64 and copied to the
 * current device; for N <= 256 the multiplier tables of
 * SQ_OPT_MULTIPLIER_TABLE are built there too (synchronous). */
int sq_precond_setup(int N, int rank, sq_precond **out);
/* The exponential-sum nodes t[r] and weights w[r], r < rank (host arrays,
 * either may be NULL; nothing is written for rank 0). SQ_EINVAL for a
 * preconditioner that is not an exponential sum. */
int sq_precond_factors(const sq_precond *p, double *t, double *w);

/* A rank-R canonical preconditioner from given factors (Sec. 4.2, Eq. 34 in
 * general form): G(k1,k2,k3) = sum_r f1[r N + k1] f2[r N + k2] f3[r N + k3]
 * on every nonzero mode (k1 on the slowest grid axis x1), G(0,0,0) = 0. f1,
 * f2, f3: HOST arrays of R x N doubles, read during the call; f2 or f3 NULL
 * repeats f1. Every factor row must be even, f[r N + k] = f[r N + N - k]
 * (within 1e-12 of the row's largest entry): G is then a function of the
 * per-axis eigenvalues l_k, the class the separable Hartley transform
 * diagonalises. 1 <= R <= 256; SQ_EINVAL otherwise (N as for
 * sq_precond_setup). Synchronous, like sq_precond_setup. */
int sq_precond_setup_canonical(int N, int R, const double *f1, const double *f2, const double *f3,
                               sq_precond **out);

/* The paper's construction of the canonical factors (Sec. 4.2): a Tucker
 * decomposition of G+ with multilinear rank (r, r, r) -- the higher-order
 * SVD (De Lathauwer, De Moor & Vandewalle 2000; the paper computes it with a
 * multigrid acceleration), which for the symmetric G+ uses one even factor
 * for all modes -- then Tucker-to-canonical: each mode-3 slice of the r^3
 * core is eigen-decomposed, giving up to r^2 terms sigma (U e) (x) (U e) (x)
 * U[:, c]; terms with |sigma| <= tol * max|sigma| are dropped (tol = 0 keeps
 * all r^2 and reproduces the Tucker tensor). 1 <= r <= min(N/2 + 1, 64),
 * 0 <= tol < 1, and the resulting rank must be <= 256; SQ_EINVAL otherwise.
 * Host-side FP64 setup (O(N^4 / 16) flops for the Gram matrix), then
 * synchronous upload. */
int sq_precond_setup_tucker(int N, int r, double tol, sq_precond **out);

/* Canonical rank of p (0 for the exact diagonal) and max over the nonzero
 * modes of |(l_k1 + l_k2 + l_k3) G(k) - 1| (the preconditioner's relative
 * error; 0 for the exact diagonal). Either output may be NULL; the error is
 * evaluated on the host in O(R N^3 / 8). */
int sq_precond_info(const sq_precond *p, int *rank, double *max_rel_err);
void sq_precond_destroy(sq_precond *p);

/* Scratch fields for one solve at grid N and the given precision (device
 * memory, allocated here with cudaMalloc): SQ_FP64 4 N^3 doubles, SQ_FP32_REFINE
 * 5 N^3 floats, plus reduction partials. One workspace serves one solve at a
 * time: solves that share it must be ordered on one stream. */
int sq_workspace_create(int N, int precision, sq_workspace **out);
void sq_workspace_destroy(sq_workspace *w);

/* PCG solve of A psi = b_dir (dir = 0,1,2 for e_1,e_2,e_3) on the zero-mean
 * subspace (Eqs. 24-25), preconditioned by `pc` (Sec. 4.2). Hestenes-Stiefel
 * recurrence, x0 = x0 if given (device, N^3 doubles) else 0; stops when
 * ||r||_2/||b||_2 <= tol on the recurrence residual, then confirms on the true
 * FP64 residual (continuing from the current iterate if that fails). The
 * result psi (device, N^3 doubles, may alias x0) is projected to zero mean.
 * SQ_FP32_REFINE: psi is refined in FP64, each correction solved in FP32 to
 * relative residual 1e-5 by default (SQ_OPT_INNER_TOL_EXP; at most max_iter
 * inner iterations in total). Returns SQ_OK, SQ_ENOCONV (tolerance missed
 * within max_iter; psi and info are valid) or SQ_ETIMEOUT: a bounded device
 * wait (pass E's staging of p and x in the FP32 iteration, SQ_OPT_WAIT_POLLS)
 * gave up; that kernel read its operands from global memory instead, the
 * solve ran to the end, and psi (zero mean) and info are complete as for
 * SQ_OK. Synchronizes `stream` (the host checks convergence). info may be
 * NULL. */
int sq_pcg_solve(const sq_coeffs *c, const sq_precond *pc, sq_workspace *w, int dir, double tol,
                 int max_iter, int precision, const double *x0, double *psi,
                 sq_solve_info *info, sq_stream_t stream);

/* Batched solves: many independent corrector problems (realizations x
 * right-hand sides, any mix of grid sizes) advanced together, each kernel
 * launch covering every solve. Precision as SQ_FP32_REFINE. */
typedef struct sq_batch sq_batch;

typedef struct sq_solve_desc {
  const sq_coeffs *coeffs; /* realization; must outlive the batch              */
  int dir;                 /* right-hand side e_{dir+1}, 0..2                   */
  double *psi;             /* device, N^3 doubles: the solution (zero mean)     */
} sq_solve_desc;

/* Tile shape per grid size; an entry sets every field for its N, and 0
 * restores that field's default. Hartley-pass tile of `dht_pencils`
 * complex pencils (a power of two, 2*dht_pencils dividing N), operator work
 * items of `stencil_planes` x1-planes (register kernels; for the staged
 * kernel, the planes each block marches, at least 4; its default fills one
 * wave of blocks), the FP32 operator
 * variant of single solves `stencil_rows` (1, 2, 4 node rows per thread, or 8
 * for the shared-memory-staged kernel; see SQ_OPT_STENCIL_ROWS; batches use
 * 1), and `dht_pencils_e`, the tile of the last FP32 pass of a PCG iteration
 * (x3 transform with the x and p updates, which stages p and x in shared
 * memory; 0 = dht_pencils; single solves only). */
typedef struct sq_tile_config {
  int N;
  int dht_pencils;
  int stencil_planes;
  int stencil_rows;
  int dht_pencils_e;
} sq_tile_config;

/* Process-wide tile choice per grid size for single solves (FP32 Hartley
 * passes and the operator of both precisions) and the default of new batches;
 * ntiles = 0 restores the built-in defaults. Not thread-safe with concurrent
 * solves. */
int sq_set_tiles(const sq_tile_config *tiles, int ntiles);

/* Process-wide switches (not thread-safe with concurrent solves).
 * SQ_OPT_STRIDED_TWO_STAGE (default 1): the FP32 Hartley passes (x1/x2 and the
 * contiguous x3) use the two-stage plans (one register stage from global
 * memory, one in-place shared-memory stage, an all-thread combine) where N
 * allows (16, 32, 64, 128, 256) and the tile has 8 or 16 pencils; 0 selects
 * the generic shared-memory Stockham tile everywhere. 2 is accepted and acts
 * as 1. FP64 passes (ALU-bound; the two-stage plans measured slower there)
 * always use the generic tile.
 * SQ_OPT_STENCIL_ROWS (default 0 = automatic, i.e. 8): the FP32 operator of
 * single solves for grid sizes without a per-N choice
 * (sq_tile_config.stencil_rows): 1, 2 or 4 node rows per thread with a
 * register plane queue (used where N is divisible by it, else the next
 * smaller), or 8: planes staged through shared memory with asynchronous
 * copies (where N is a multiple of 32 and p is 16-byte aligned, else 4).
 * Results are identical up to the order of the p.Ap summation.
 * SQ_OPT_INNER_TOL_EXP (default 5): each inner FP32 solve of SQ_FP32_REFINE
 * (single and batched) cuts its residual by 10^-value, or just enough for the
 * outer tolerance when that is less; 2 <= value <= 7.
 * SQ_OPT_WAIT_POLLS (default 4194304 = 2^22): how many times the FP32 pass E
 * of single solves polls the barrier of its bulk copies of p and x before it
 * gives up, reads them from global memory, flags the solve (SQ_ETIMEOUT) and
 * stops staging; 0 gives up at once. The block still waits (up to 2^24 polls)
 * for its copies in flight before it exits. 0 <= value <= 2^24.
 * SQ_OPT_MULTIPLIER_TABLE (default 1): preconditioners of grids N <= 256 carry
 * their multiplier G tabulated (built on the device by sq_precond_setup* from
 * the same factors, summed in FP64): (N/2 + 1)^3 FP64 values on the
 * mirror-reduced modes, and an FP32 copy of (N/2 + 1)^2 N values. The x1 pass
 * of single solves reads G from it (FP32: each tile's slice prefetched into
 * shared memory) instead of summing the canonical terms (or dividing, for the
 * exact diagonal in FP64) per mode; 0 evaluates G on the fly. FP32 passes
 * with the exact diagonal and batches always evaluate it on the fly. Results
 * agree to rounding.
 * SQ_OPT_CONV_TC (default 1): the warm-start net's 32 -> 32 channel
 * convolutions (forward and data gradient) and the output layer's forward
 * convolution (32 -> 3 channels, 16 accumulator columns) run on the
 * 5th-generation tensor cores as direct convolutions: the input halo of a tile of 8 x 16 x D output
 * voxels is staged once in shared memory and every tap's A operand is that
 * halo read through a shifted descriptor (tcgen05.mma, M = 128 voxels, N = 32,
 * K = 16, FP32 accumulator in tensor memory; bounded waits: a wait that gives
 * up makes sq_net_predict / sq_net_train_step return SQ_ETIMEOUT). 1 picks
 * the tile depth D in {2, 4} from the tile count, 2 or 4 fixes it; 0 uses the
 * mma.sync kernels. Results agree to FP32 rounding of the same BF16 inputs.
 * SQ_OPT_PCG_GRAPHS (default 1): sq_pcg_solve replays a CUDA graph of two
 * PCG iterations (twelve kernels; eight for sq2d_pcg_solve) per host step
 * instead of launching each kernel, captured on first use for the solve's
 * fields, coefficients,
 * preconditioner and options, and kept in the workspace (up to 8 graphs;
 * any sq_set_option or sq_set_tiles call makes later solves capture anew).
 * While profiling is enabled, or when the stream is being captured by the
 * caller, kernels are launched one by one. 0 always launches them one by
 * one. Results are identical.
 */
enum sq_option {
  SQ_OPT_STRIDED_TWO_STAGE = 1,
  SQ_OPT_STENCIL_ROWS = 2,
  SQ_OPT_INNER_TOL_EXP = 3,
  SQ_OPT_WAIT_POLLS = 4,
  SQ_OPT_MULTIPLIER_TABLE = 5,
  SQ_OPT_CONV_TC = 6,
  SQ_OPT_PCG_GRAPHS = 7
};
int sq_set_option(int key, int value);

/* Plans a batch of `count` solves; precs[k] is the preconditioner (same N) of
 * descs[k]. Allocates 5 N^3 floats per solve plus scalars and partials, and
 * captures the batched inner PCG iteration into a CUDA graph on first solve.
 * tiles (ntiles entries, may be NULL) overrides the default tile per N.
 * Synchronous. */
int sq_batch_create(int count, const sq_solve_desc *descs, const sq_precond *const *precs,
                    const sq_tile_config *tiles, int ntiles, sq_batch **out);
void sq_batch_destroy(sq_batch *b);

/* Solves every problem of the batch to ||b - A psi||/||b|| <= tol (FP64 true
 * residual), x0 = 0, at most max_iter inner iterations per solve. infos (host,
 * `count` entries, may be NULL) receives per-solve iterations and residuals.
 * Returns SQ_ENOCONV if any solve missed the tolerance. Synchronizes `stream`. */
int sq_pcg_solve_batched(sq_batch *b, double tol, int max_iter, sq_solve_info *infos, sq_stream_t stream);

/* Homogenized matrix (Sec. 3.4, Eqs. 21-23) from the three correctors psi_i
 * (device, N^3 doubles each):
 *   A_hom[3*i+j] = delta_ij mean(a_j) + mean(a_j * D_j psi_i)   (edge form)
 * and, if A_energy != NULL, the symmetric energy form
 *   A_energy[3*i+j] = mean(sum_d a_d (delta_id + D_d psi_i)(delta_jd + D_d psi_j)).
 * Outputs are HOST arrays of 9 doubles. Synchronizes `stream`. */
int sq_homogenized_matrix(const sq_coeffs *c, const double *psi0, const double *psi1,
                          const double *psi2, double *A_hom, double *A_energy, sq_stream_t stream);

/* Ensemble statistics of the homogenized matrix (Sec. 5, Eq. A_hom_Empir and
 * the sample standard deviation sigma^M_L estimating Eq. var): for the M >= 2
 * realizations seeds[0..M) of the L^3 checkerboard (cells as sq_build_coeffs
 * with p_hi, a_lo, a_hi), solves the three correctors of each with the batched
 * solver (FP32 PCG in FP64 refinement to `tol`, preconditioner `rank`, at most
 * max_iter inner iterations), takes the edge-form A_hom of each, and returns
 * on the host, entry-wise (row-major 3 x 3):
 *   mean[9]  = (1/M) sum_m A^(m),
 *   sigma[9] = sqrt( sum_m (A^(m) - mean)^2 / (M - 1) ),
 * and, where not NULL, per_real[9 M] (realization m at 9 m) and iters[3 M]
 * (inner iterations of corrector i of realization m at 3 m + i).
 * Realizations are solved `chunk` at a time (0 = all at once; device memory
 * about 84 N^3 bytes per realization of a chunk). Returns SQ_ENOCONV (with
 * all outputs filled) if a solve missed the tolerance. Synchronous. */
int sq_ensemble_ahom(int L, int n, const uint64_t *seeds, int M, double p_hi, double a_lo, double a_hi,
                     int rank, double tol, int max_iter, int chunk, double *mean, double *sigma,
                     double *per_real, int *iters, sq_stream_t stream);

/* Learned warm start (an addition to the paper's method): a periodic 3D
 * convolutional net -- 6 layers of 3x3x3 convolutions, 32 channels, GELU,
 * BF16 weights and activations with FP32 accumulation on the tensor cores --
 * maps the coefficient field (+1 high / -1 low per grid voxel) to a first
 * guess of the three correctors psi_1..3 (scaled by out_scale). The guess is
 * passed to sq_pcg_solve as x0; the solve keeps it only if it lowers the
 * residual. Grids N = 32, 64, 96 or 128 (N % 32 == 0). */
typedef struct sq_net sq_net;

/* Creates the net for grid N with buffers for up to max_batch training
 * samples; weights He-normal from `seed` (SplitMix64), biases zero. */
int sq_net_create(int N, int max_batch, uint64_t seed, double out_scale, sq_net **out);
void sq_net_destroy(sq_net *net);
/* FP32 parameters (per layer: weights [27][cout][cin], then bias [cout]):
 * copy out (host may be NULL to query *count) or in (resets the optimizer). */
int sq_net_params(const sq_net *net, float *host, int64_t *count);
int sq_net_set_params(sq_net *net, const float *host, int64_t count);
/* Gradient of the last sq_net_train_step (same layout as the parameters). */
int sq_net_grads(const sq_net *net, float *host, int64_t count);
/* Guess for the three correctors of realization c (device outputs, N^3 doubles
 * each). Asynchronous on `stream`, except with SQ_OPT_CONV_TC = 1, where it
 * synchronizes `stream` to read back the tensor-core kernels' status
 * (SQ_ETIMEOUT if a bounded wait gave up). */
int sq_net_predict(sq_net *net, const sq_coeffs *c, double *psi0, double *psi1, double *psi2,
                   sq_stream_t stream);
/* One Adam step (lr; beta 0.9 / 0.999) against the targets targets[3*b + i]
 * (device, N^3 doubles: psi_i of sample b) for the `batch` realizations
 * cs[b], with e = (prediction - target) / out_scale and loss_type 0: mean of
 * e^2; 1: mean of e . A e (the energy norm of the error under each sample's
 * own operator -- the norm PCG reduces); 2: mean of r . r with r =
 * (A prediction - b_i) / out_scale (the residual norm the solver's stopping
 * rule measures; the targets are not read, but must be valid pointers).
 * *loss (host, may be NULL) receives that loss for the forward pass
 * (synchronizes `stream`). */
int sq_net_train_step(sq_net *net, int batch, const sq_coeffs *const *cs, const double *const *targets,
                      float lr, int loss_type, double *loss, sq_stream_t stream);

/* A_hom without allocating: for callers that may not allocate device memory
 * when they need the result (code running under CUDA stream capture, or a
 * framework that hands out all device memory from its own pool). The paper has
 * no counterpart; the arithmetic is that of sq_homogenized_matrix. Inputs are
 * device pointers the caller owns: `phase` (L^3 bytes, nonzero = a_hi, index
 * c3 + L*c2 + L*L*c1) and the three correctors psi_i (N^3 doubles, N = L*n).
 * Output: `out` (device, 18 doubles) = A_hom[9] (edge form, row-major) then
 * the energy form[9]. Sizes as for sq_build_coeffs (N <= 512), else SQ_EINVAL.
 * Asynchronous on `stream`; calls no allocator. Its reduction scratch is one
 * fixed 2.36 MB __device__ array per GPU, held until the process exits and
 * shared by every call: calls that overlap on the GPU race, so order them on
 * one stream. The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) with that device current: make it before any stream
 * capture. */
int sq_homogenized_matrix_noalloc(int L, int n, const uint8_t *phase, double a_lo, double a_hi,
                                  const double *psi0, const double *psi1, const double *psi2,
                                  double *out, sq_stream_t stream);

/* Building blocks, exposed for verification (asynchronous):
 * y = A x (FP64 or FP32 fields), b = b_dir, z = G-preconditioned r (the full
 * 3D transform pipeline of the solver; w must match pc's N and the field type:
 * an SQ_FP64 workspace for the double version, SQ_FP32_REFINE for float). */
int sq_apply_operator(const sq_coeffs *c, const double *x, double *y, sq_stream_t stream);
int sq_apply_operator_f32(const sq_coeffs *c, const float *x, float *y, sq_stream_t stream);
int sq_rhs(const sq_coeffs *c, int dir, double *b, sq_stream_t stream);
int sq_apply_precond(const sq_precond *pc, sq_workspace *w, const double *r, double *z,
                     sq_stream_t stream);
int sq_apply_precond_f32(const sq_precond *pc, sq_workspace *w, const float *r, float *z,
                         sq_stream_t stream);

/* Kernel timing aid: while enabled, the library records a CUDA event pair on
 * the launching stream around each of its kernel launches and sorts them into
 * kernel classes (sq_profile_class_name). enable = 1 clears the totals and
 * starts recording, 0 stops. Not thread-safe: one host thread at a time. */
int sq_profile_enable(int enable);
/* Synchronizes the recorded events and returns the number of classes (or
 * -SQ_ECUDA); for k < min(classes, max_classes) fills ms[k] (summed device time
 * of the class) and launches[k], then clears the record. Either array may be
 * NULL. */
int sq_profile_read(double *ms, int64_t *launches, int max_classes);
/* The launches of the last sq_profile_read that did work: per class, those
 * lasting at least half of the class median (the others returned at
 * entry because their solve had already stopped, e.g. the iterations queued
 * behind the host's convergence check). Fills ms[k] and launches[k] as
 * sq_profile_read does; returns the number of classes. */
int sq_profile_work(double *ms, int64_t *launches, int max_classes);
const char *sq_profile_class_name(int k);
/* Kernel launches the single-solve path (sq_pcg_solve, sq_homogenized_matrix,
 * the coefficient and verification calls) has issued since the library was
 * loaded, whether or not profiling is enabled (a host-side counter). */
int64_t sq_launch_count(void);

/* Throughput probes (measurement aids for rooflines; the paper has no
 * counterpart). Both are synchronous on `stream`, time their own kernel with
 * CUDA events after a warm-up launch, and report the rate at the clocks of
 * that moment.
 * sq_probe_fma: precision 0 = FP64, 1 = FP32; a grid at the occupancy limit,
 * eight independent fused multiply-add chains per thread, about 30 ms of
 * work; *tflops = 2 flops per FMA / time, *ms the kernel time (either may be
 * NULL). Allocates 8 bytes per block (stream-ordered) for its guard output.
 * sq_probe_copy: dst = src over `bytes` (device buffers, 16-byte aligned,
 * bytes a multiple of 16), `reps` sweeps in one launch (1..10000); *gbps = 2 bytes reps /
 * time (read + write, as a STREAM copy). Buffers far above the L2 size measure
 * HBM; buffers that fit in L2 measure L2. */
int sq_probe_fma(int precision, double *tflops, float *ms, sq_stream_t stream);
int sq_probe_copy(const void *src, void *dst, size_t bytes, int reps, double *gbps, sq_stream_t stream);

const char *sq_strerror(int status);

/* ------------------------------------------------------------------ 2D
 * The 2D corrector problem of the paper's 2D experiments (Sec. 5): the same
 * method on an N x N periodic grid, N = L n with 8 <= N <= 2048, N even,
 * N = 2^a 3^b with b <= 1 (x2 contiguous, index j2 + N j1), two correctors
 * psi_1, psi_2 and the 2 x 2 A_hom; FP64 throughout.
 * - Cells: cell (c1, c2) of the L x L lattice is high iff the top 53 bits of
 *   SplitMix64 output number c2 + L c1 (the rule of sq_build_coeffs on its
 *   slab c1 = 0) are below floor(p_hi 2^53). Sub-cell inclusions: a centred
 *   square of side `sub` grid intervals per cell (sq2d_coeffs_set_subcell).
 * - Operator: sum_d D_d^T diag(a_d) D_d with a_d(j) the mean of the two
 *   voxels beside the edge j -> j + e_d; RHS b_i(j) = a_i(j) - a_i(j - e_i).
 * - Preconditioner: G(k1, k2) = 1/(l_k1 + l_k2), G(0, 0) = 0 (rank 0), or
 *   the rank-R exponential sum sum_r w_r exp(-t_r (l_k1 + l_k2)), 2 <= R <= 64,
 *   fitted on the 2D spectrum; applied as a 2D Hartley transform.
 * Handles, ownership, streams and errors as for the 3D calls. */
typedef struct sq2d_coeffs sq2d_coeffs;
typedef struct sq2d_precond sq2d_precond;
typedef struct sq2d_workspace sq2d_workspace;

int sq2d_build_coeffs(int L, int n, uint64_t seed, double p_hi, double a_lo, double a_hi, sq_stream_t stream,
                      sq2d_coeffs **out);
/* L^2 phases in HOST memory (0 = a_lo, nonzero = a_hi, index c2 + L c1). */
int sq2d_coeffs_from_host(int L, int n, const uint8_t *host_phase, double a_lo, double a_hi, sq_stream_t stream,
                          sq2d_coeffs **out);
/* 1 <= sub <= n with n - sub even (sub = n: whole cells). */
int sq2d_coeffs_set_subcell(sq2d_coeffs *c, int sub);
/* Copies the L^2 phases to host_phase (synchronous). */
int sq2d_coeffs_cells(const sq2d_coeffs *c, uint8_t *host_phase);
void sq2d_coeffs_destroy(sq2d_coeffs *c);

int sq2d_precond_setup(int N, int rank, sq2d_precond **out);
/* Exponential-sum nodes and weights (rank entries each; NULL allowed). */
int sq2d_precond_factors(const sq2d_precond *p, double *t, double *w);
void sq2d_precond_destroy(sq2d_precond *p);

/* 4 N^2 doubles of scratch plus reduction buffers (device). */
int sq2d_workspace_create(int N, sq2d_workspace **out);
void sq2d_workspace_destroy(sq2d_workspace *w);

/* PCG for corrector dir (0 or 1) to ||b - A psi|| <= tol ||b|| from psi = 0;
 * psi: DEVICE array of N^2 doubles, zero-mean on return. SQ_ENOCONV if the
 * tolerance is not met within max_iter. */
int sq2d_pcg_solve(const sq2d_coeffs *c, const sq2d_precond *pc, sq2d_workspace *w, int dir, double tol,
                   int max_iter, double *psi, sq_solve_info *info, sq_stream_t stream);
/* A_hom (edge form, row-major 2 x 2) and, if A_energy is not NULL, the
 * energy form, from the two correctors (DEVICE arrays; synchronous on the
 * handle's stream). */
int sq2d_homogenized_matrix(const sq2d_coeffs *c, const double *psi0, const double *psi1, double *A_hom,
                            double *A_energy);
/* Verification blocks (DEVICE arrays of N^2 doubles): y = A x; b = b_dir;
 * z = G-preconditioned r (zero mean). */
int sq2d_apply_operator(const sq2d_coeffs *c, const double *x, double *y, sq_stream_t stream);
int sq2d_rhs(const sq2d_coeffs *c, int dir, double *b, sq_stream_t stream);
int sq2d_apply_precond(const sq2d_precond *pc, sq2d_workspace *w, const double *r, double *z, sq_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SQ_H */
