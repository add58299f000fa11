// Internal declarations shared by the libsq translation units.
//
// Field layout (Sec. 3.2, big-endian order): node (j1,j2,j3) of the N^3 grid at
// j3 + N*j2 + N*N*j1. Cells: (c1,c2,c3) at c3 + L*c2 + L*L*c1, c = j / n.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sq.h"

namespace sq {

constexpr int kThreads = 256;        // block size of every field kernel
constexpr int kMaxPartials = 16384;  // max blocks of a reducing kernel
constexpr int kPollChunk = 2;        // PCG iterations launched per host poll of the stop flag
constexpr int kMaxQ = 24;            // max quantities reduced by one kernel
constexpr int kMaxN = 512;
constexpr int kMaxRank = 256;    // canonical terms of a preconditioner from given factors
constexpr int kMaxExpRank = 64;  // terms of the exponential-sum preconditioner

// Device-resident solver scalars. Written only by the last block of a
// reducing kernel (or by the host before a solve), read by later kernels.
struct Scalars {
  double bb;        // ||b||^2
  double rr;        // ||r||^2 of the recurrence residual
  double rz;        // r.z (current)
  double rz_old;    // r.z (previous iteration)
  double pq;        // p.Ap
  double alpha;     // alpha_k = rz / pq
  double beta;      // beta_k = rz_new / rz_old
  double tol2;      // tol^2 * bb
  double tolrel2;   // tol^2 (set by the host before a solve)
  double mean;      // mean of the final iterate
  double rr_true;   // ||b - A x||^2 recomputed
  double red[kMaxQ];  // raw sums of the last reduction (verification / A_hom)
  int done;         // 1: no further PCG kernel does work
  int conv;         // 1: converged (0 with done=1: max_iter or breakdown)
  int iter;         // x updates so far (cumulative over restarts)
  int max_iter;
  int x_pending;    // 1: x += alpha p of the last iteration not applied yet
  int breakdown;    // 1: non-positive p.Ap or r.z
  unsigned int ticket;  // last-block counter (reset by the last block)
  int fault;            // 1: a bounded device wait gave up (the kernel fell back; reported as SQ_ETIMEOUT)
};

enum FinalizeOp : int {
  FIN_NONE = 0,      // raw sums -> red[]
  FIN_ALPHA = 1,     // q = A p: pq = s0, alpha = rz / pq
  FIN_RESID = 2,     // r = b - A x: rr = s0, bb = s1 (if set_bb), done if rr <= tol2
  FIN_RR_ITER = 3,   // r -= alpha q: rr = s0, iter++, convergence / max_iter check
  FIN_RZ_FIRST = 4,  // r.z of the initial residual
  FIN_RZ_BETA = 5,   // r.z -> beta
  FIN_MEAN = 6,      // sum(x) -> mean
};

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

// ---------------------------------------------------------------- reductions

// Per-thread partial sums. FP64 kernels accumulate in FP64. FP32 kernels use
// compensated (Kahan) FP32 sums per thread and carry them on as float-float
// numbers (below) through the warp, block and last-block sums, converting to
// FP64 once, for the final scalar: GB300's FP64 pipe runs at ~1/58 of its FP32
// rate, and even a handful of FP64 adds per warp in every block of an FP32
// pass costs more pipe time than the pass's own arithmetic.
template <typename T>
struct Accum;

// Float-float (double-word) value hi + lo, |lo| <= ulp(hi)/2. The sum of two
// is Knuth's TwoSum of the high parts (exact error term), plus the low parts,
// renormalised by Dekker's Fast2Sum (Dekker 1971; the "sloppy" double-word
// addition). Relative error ~2^-44 per addition, with FP32 instructions only.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_renorm(float s, float e) {
  const float h = s + e;
  return FF{h, e - (h - s)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bv = s - a.hi;
  float e = (a.hi - (s - bv)) + (b.hi - bv);
  e += a.lo + b.lo;
  return ff_renorm(s, e);
}

template <>
struct Accum<double> {
  using Part = double;
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ double part() const { return s; }
};
template <>
struct Accum<float> {
  using Part = FF;
  float s = 0.f, c = 0.f;  // running sum and its compensation (sum = s - c)
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ void add_prod(float a, float b) { add(a * b); }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
  // |c| <= ulp(s) after every step, so Fast2Sum's precondition holds
  __device__ __forceinline__ FF part() const { return ff_renorm(s, -c); }
};

// Operations on a partial sum (double or FF) used by the block reductions.
__device__ __forceinline__ double part_zero(double) { return 0.0; }
__device__ __forceinline__ FF part_zero(FF) { return FF{0.f, 0.f}; }
__device__ __forceinline__ double part_add(double a, double b) { return a + b; }
__device__ __forceinline__ FF part_add(FF a, FF b) { return ff_add(a, b); }
__device__ __forceinline__ double part_shfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ FF part_shfl(FF v, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double part_value(double v) { return v; }
__device__ __forceinline__ double part_value(FF v) { return (double)v.hi + (double)v.lo; }
// A partial occupies one 8-byte slot of the partials buffer either way.
__device__ __forceinline__ void part_store(double *p, double v) { *p = v; }
__device__ __forceinline__ void part_store(double *p, FF v) {
  *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ double part_load(const double *p, double) { return __ldcg(p); }
__device__ __forceinline__ FF part_load(const double *p, FF) {
  const float2 f = __ldcg(reinterpret_cast<const float2 *>(p));
  return FF{f.x, f.y};
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename P>
__device__ __forceinline__ P warp_sum_part(P v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = part_add(v, part_shfl(v, o));
  return v;
}

// Block-reduces NQ per-thread values, writes one partial per block and lets
// the last block to finish sum all partials in a fixed order (deterministic,
// independent of which block is last). Returns true in every thread of that
// last block; the sums are then in out[0..NQ). Requires blockDim = kThreads.
// P is double or FF; the sums stay in P until the final conversion.
// The explicit form takes the block's index `bid` among the `nblk` blocks that
// share one ticket, and the partials row stride `pstride` (batched kernels
// reduce per solve); reduce_last_block uses the whole grid.
template <int NQ, typename P>
__device__ __forceinline__ bool reduce_last_block_ex(P (&v)[NQ], double *partials, int pstride, unsigned *ticket,
                                                     int nblk, int bid, double (&out)[NQ]) {
  __shared__ P s_w[NQ][kThreads / 32];
  __shared__ unsigned s_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, wid = tid >> 5;
  const P z = part_zero(v[0]);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    P s = warp_sum_part(v[q]);
    if (lane == 0) s_w[q][wid] = s;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      P s = z;
      for (int w = 0; w < kThreads / 32; ++w) s = part_add(s, s_w[q][w]);
      part_store(&partials[q * pstride + bid], s);
    }
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == (unsigned)(nblk - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    P s = z;
    for (int i = tid; i < nblk; i += kThreads) s = part_add(s, part_load(&partials[q * pstride + i], z));
    s = warp_sum_part(s);
    if (lane == 0) s_w[q][wid] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    P s = z;
    for (int w = 0; w < kThreads / 32; ++w) s = part_add(s, s_w[q][w]);
    out[q] = part_value(s);
  }
  if (tid == 0) *ticket = 0u;
  return true;
}

template <int NQ, typename P>
__device__ __forceinline__ bool reduce_last_block(P (&v)[NQ], double *partials, unsigned *ticket,
                                                  double (&out)[NQ]) {
  const int nblk = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  return reduce_last_block_ex<NQ>(v, partials, kMaxPartials, ticket, nblk, bid, out);
}

// Scalar bookkeeping done by thread 0 of the last block.
__device__ __forceinline__ void finalize_scalars(Scalars *st, int op, const double *s, int nq) {
  for (int q = 0; q < nq && q < kMaxQ; ++q) st->red[q] = s[q];
  switch (op) {
    case FIN_ALPHA:
      st->pq = s[0];
      if (s[0] > 0.0 && st->rz > 0.0) {
        st->alpha = st->rz / s[0];
      } else {
        st->alpha = 0.0;
        st->done = 1;
        st->breakdown = 1;
      }
      break;
    case FIN_RESID:
      st->bb = s[1];
      st->tol2 = st->tolrel2 * s[1];
      st->rr = s[0];
      st->rr_true = s[0];
      st->done = (s[0] <= st->tol2 || !(s[1] > 0.0)) ? 1 : 0;
      st->conv = st->done;
      st->x_pending = 0;
      break;
    case FIN_RR_ITER:
      st->rr = s[0];
      st->iter += 1;
      if (s[0] <= st->tol2) {
        st->done = 1;
        st->conv = 1;
        st->x_pending = 1;
      } else if (st->iter >= st->max_iter || !(s[0] == s[0])) {
        st->done = 1;
        st->x_pending = 1;
      }
      break;
    case FIN_RZ_FIRST:
      st->rz = s[0];
      if (!(s[0] > 0.0)) { st->done = 1; st->breakdown = 1; }
      break;
    case FIN_RZ_BETA:
      st->rz_old = st->rz;
      st->rz = s[0];
      if (s[0] > 0.0) {
        st->beta = s[0] / st->rz_old;
      } else {
        st->beta = 0.0;
        st->done = 1;
        st->breakdown = 1;
      }
      break;
    default:
      break;
  }
}

// ------------------------------------------------------------ host launchers

// Multi-level media (varying contrast): a cell's phase byte v selects level
// min(v, K - 1) of K <= kMaxLevels coefficient values.
constexpr int kMaxLevels = 4;
constexpr int kMaxLayers = kMaxLevels - 1;

struct CellsDev {
  const uint8_t *phase;  // L^3 cell phases (levels)
  int L, n, N;
  double a_lo, a_hi;  // values of levels 0 and 1
  // Sub-cell inclusions (Sec. 3.1): a voxel at cell-local index u (per axis)
  // takes its cell's value only if sub_lo <= u < sub_hi on every axis, else
  // a_lo. The default is the whole cell (the checkerboard).
  int sub_lo = 0, sub_hi = 1 << 30;
  // Levels above 1 (host side; K = 2 + the count set): a_up[l - 2] = value of level l.
  double a_up[kMaxLevels - 2] = {0.0, 0.0};
  // Threshold layers: the value of a voxel at level v is
  //   a_lo + sum_{l = 1 .. K-1} [v >= l] (value(l) - value(l - 1)),
  // and an edge coefficient is the mean of its four voxels, so it is the sum
  // over layers l of the layer's table at k_l = the number of the four voxels
  // with level >= l. Layer 0 (l = 1): a_edge = (k a_hi + (4-k) a_lo)/4; a
  // higher layer adds k (value(l) - value(l - 1))/4. A node's six edges touch
  // 24 voxel slots, K_l of them at level >= l: the diagonal is the same sum
  // with 24 in place of 4. The tables are filled on the host (fill_tables);
  // two-level media use layer 0 only.
  int layers = 1;  // K - 1
  double edge_d[kMaxLayers][5], diag_d[kMaxLayers][25];
  float edge_f[kMaxLayers][5], diag_f[kMaxLayers][25];
};

// Anything but the plain two-level checkerboard of whole cells.
inline bool general_media(const CellsDev &c) { return c.layers > 1 || c.sub_lo != 0 || c.sub_hi < (1 << 30); }

inline double level_value(const CellsDev &c, int l) { return l == 0 ? c.a_lo : l == 1 ? c.a_hi : c.a_up[l - 2]; }

inline void fill_tables(CellsDev &c) {
  for (int l = 0; l < kMaxLayers; ++l) {
    const double lo = (l == 0) ? c.a_lo : 0.0;
    const double step = (l < c.layers) ? level_value(c, l + 1) - level_value(c, l) : 0.0;
    for (int k = 0; k <= 4; ++k) {
      c.edge_d[l][k] = (l == 0) ? (k * c.a_hi + (4 - k) * lo) * 0.25 : k * step * 0.25;
      c.edge_f[l][k] = (float)c.edge_d[l][k];
    }
    for (int k = 0; k <= 24; ++k) {
      c.diag_d[l][k] = (l == 0) ? (k * c.a_hi + (24 - k) * lo) * 0.25 : k * step * 0.25;
      c.diag_f[l][k] = (float)c.diag_d[l][k];
    }
  }
}

// Shared-memory bytes of the pattern tables of `layers` layers.
template <typename T>
constexpr size_t tab_bytes(int layers) {
  return (size_t)layers * 256 * 9 * sizeof(T);
}

template <typename T>
__device__ __forceinline__ const T *edge_table(const CellsDev &c, int l);
template <>
__device__ __forceinline__ const double *edge_table<double>(const CellsDev &c, int l) { return c.edge_d[l]; }
template <>
__device__ __forceinline__ const float *edge_table<float>(const CellsDev &c, int l) { return c.edge_f[l]; }
template <typename T>
__device__ __forceinline__ const T *diag_table(const CellsDev &c, int l);
template <>
__device__ __forceinline__ const double *diag_table<double>(const CellsDev &c, int l) { return c.diag_d[l]; }
template <>
__device__ __forceinline__ const float *diag_table<float>(const CellsDev &c, int l) { return c.diag_f[l]; }

struct RedBuf {
  Scalars *st;
  double *partials;  // kMaxQ * kMaxPartials
};

// stencil.cu
// thr[0..2]: level thresholds on the top 53 bits (see k_coeff_gen).
cudaError_t launch_coeff_gen(uint8_t *phase, int L, uint64_t seed, const uint64_t *thr, cudaStream_t s);
// The same draw for cells 0 .. ncell-1 (a 2D lattice: ncell = L^2).
cudaError_t launch_coeff_gen_cells(uint8_t *phase, int ncell, uint64_t seed, const uint64_t *thr, cudaStream_t s);
cudaError_t allow_dynamic_smem(const void *kern, size_t smem);
enum StencilMode : int { ST_MATVEC = 0, ST_RESID = 1, ST_RHS = 2 };
// y = A x (ST_MATVEC, reduces x.y), y = b_dir - A x (ST_RESID, reduces ||y||^2
// and ||b||^2), y = b_dir (ST_RHS, reduces ||b||^2). Ti: type of x and of the
// arithmetic; To: type of y.
template <typename Ti, typename To>
cudaError_t launch_stencil(const CellsDev &c, int mode, int dir, const Ti *x, To *y, RedBuf rb, int fin,
                           bool check_done, cudaStream_t s);
// energy: also the six sums of the energy form (quantities 12..17)
cudaError_t launch_ahom(const CellsDev &c, const double *p0, const double *p1, const double *p2, RedBuf rb,
                        bool energy, cudaStream_t s);
template <typename T>
cudaError_t launch_x_final_sum(T *x, const T *p, RedBuf rb, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_sub_mean(T *x, RedBuf rb, long long n, cudaStream_t s);
// x64 += d32 (refinement update), and plain casts
cudaError_t launch_add_f32_to_f64(double *x, const float *d, long long n, cudaStream_t s);

// dht.cu
struct SpectralDev {
  int N;
  int rank;          // 0 = exact
  int nst;           // FFT stages
  int radix[12];
  const void *tw;    // N complex twiddles exp(-2 pi i m / N), type Cx<T>
  const void *lam;   // N eigenvalues lambda_k (T)
  // canonical factors (T), 3 x rank x N: the x1, x2 and x3 factors of term r
  // at u + (a rank + r) N, a = 0, 1, 2, each scaled by (64 N^3)^(-1/3), so
  // that G(k1,k2,k3) = sum_r u1_r(k1) u2_r(k2) u3_r(k3). Every factor is even
  // (u(k) = u(N - k)): G is then diagonal in the separable Hartley basis.
  const void *u;
  double scale;      // 1 / (64 N^3) for the exact diagonal
  // The multiplier itself, tabulated (T) times the factor pass C applies per
  // mode (FP64 8 G, FP32 2 G; see dht_tile), scale folded in as above, G(0,0,0) = 0, with m = min(k, N - k)
  // (G is even in each index) and H = N/2 + 1:
  // FP64 at gtab[(m1 H + m2) H + m3]; FP32 at gtab[(m1 H + m2) N + k3] (the
  // x3 index unreduced, so that a tile's 2P columns are one aligned run).
  // nullptr: pass C evaluates G from lam or u on the fly.
  const void *gtab = nullptr;
};
// Grids up to this size carry the multiplier tables (FP64 17 MB, FP32 17 MB
// at N = 256, resident in L2 while pass C reads them).
constexpr int kGtabMaxN = 256;
__host__ __device__ constexpr int mirror_index(int k, int N) { return k <= N - k ? k : N - k; }
enum DhtPass : int { PASS_A_RESID = 0, PASS_A_PLAIN = 1, PASS_B = 2, PASS_C = 3, PASS_E_PCG = 4, PASS_E_PLAIN = 5, PASS_D = 6 };
// One pencil pass of the 3D Hartley transform pipeline (see dht.cu).
template <typename T>
cudaError_t launch_dht_pass(int pass, const SpectralDev &sp, const T *in, T *out, T *r, const T *q, T *p, T *x,
                            RedBuf rb, bool first, bool check_done, cudaStream_t s);
int dht_tile_pencils(int N, int elem_bytes);
// The same passes on an N x N field (see dht.cu): PASS_A_*, PASS_C, PASS_E_*.
template <typename T>
cudaError_t launch_dht_pass_2d(int pass, const SpectralDev &sp, const T *in, T *out, T *r, const T *q, T *p, T *x,
                               RedBuf rb, bool first, bool check_done, cudaStream_t s);
// tile overrides (0 = default); return 0 on success
int set_dht_pencils_override(int N, int P);
int set_dht_pencils_e_override(int N, int P);  // pass E (FP32, PCG update) only
int set_stencil_planes_override(int N, int zc);
int set_stencil_rows(int rpt);  // FP32 operator rows per thread: 0 auto, 1, 2, 4
int set_stencil_rows_override(int N, int rpt);  // per grid size; 0 = the process-wide choice
int set_strided_fast(int on);  // 0: generic Stockham tiles for every pass
int set_use_gtab(int on);      // 0: pass C evaluates the multiplier on the fly everywhere
int pcg_graphs_enabled();     // single solves replay iteration graphs (SQ_OPT_PCG_GRAPHS)
int option_epoch();           // bumped by every option or tile change
int set_conv_tc(int on);       // warm-start net: 32 -> 32 convolutions on tcgen05 (1) or mma.sync (0)
int use_gtab();

// solver.cu: the kernel-event profile (sq_profile_enable) as seen by batch.cu:
// an event pair around a launch of the batch's inner iteration, or around a
// whole inner loop (a no-op index when profiling is off), whether profiling is
// on, and pausing it (true) and restoring it (false) around a graph capture.
size_t profile_begin_batch_inner(cudaStream_t s);
size_t profile_begin_batch_loop(cudaStream_t s);
void profile_end(size_t i, cudaStream_t s);
bool profile_enabled();
bool profile_pause(bool pause);
// solver.cu: read-only views of the opaque handles (used by batch.cu)
int coeffs_view(const sq_coeffs *c, CellsDev *out);
int precond_spec32(const sq_precond *p, SpectralDev *out, int *N);
// Grid sizes the solver supports: 8 <= N <= 512, N even, N = 2^a 3^b, b <= 1.
bool grid_size_ok(int N);
// Residual reduction asked of each inner FP32 solve of the refinement (10^-e).
int set_inner_tol_exp(int e);
double inner_tol();
// Polls of pass E's staging wait before it gives up (0: at once; default 2^22).
int set_stage_wait_polls(int polls);
int stage_wait_polls();
// Exponential sum sum_r w_r exp(-t_r x) ~ 1/x over the dim-D spectrum of the
// periodic Laplacian on N points per axis (dim = 2 or 3).
void exp_sum_nodes(int N, int R, int dim, std::vector<double> &t, std::vector<double> &w);
// Mixed-radix plan of the Stockham FFT of length N (returns the stage count).
int radix_plan_of(int N, int *rad);
// solver.cu: a preconditioner from host factors f (3 x R x N, unscaled; R = 0:
// the exact diagonal) and, for an exponential sum, its nodes and weights.
int precond_create(int N, int R, const double *f, const std::vector<double> &t, const std::vector<double> &w,
                   sq_precond **out);

}  // namespace sq
