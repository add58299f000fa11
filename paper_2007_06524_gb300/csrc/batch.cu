// Batched corrector solves: many independent realizations x right-hand sides,
// any mix of grid sizes, advanced together.
//
// Every kernel launch covers all solves of the batch: block b belongs to solve
// s with pre[s] <= b < pre[s+1] (binary search over the per-solve block
// counts), and each solve keeps its own device scalars, reductions (last block
// per solve, fixed summation order) and stop flag, so a converged solve costs
// only early-exiting blocks. Precision is the FP32 + FP64 scheme of
// sq_pcg_solve(SQ_FP32_REFINE): FP64 residual and update, FP32 PCG inner
// solves. The inner PCG iteration (six kernels) is captured once into a CUDA
// graph of kChunk iterations plus an active-solve count, and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <new>
#include <vector>

#include "dht_core.cuh"
#include "stencil_core.cuh"

namespace sq {

struct BSolve {
  CellsDev c;
  int dir;
  int logP;        // Hartley tile: P = 2^logP complex pencils
  int zc;          // stencil planes per block
  int nb_st;       // stencil blocks of this solve (one node row per thread)
  int in_staged;   // inner FP32 operator: 1 = staged 32 x 32 tiles (N % 32 == 0), 0 = one row per thread
  int zc_in;       // planes per block of the inner operator
  int nb_in;       // inner FP32 operator blocks of this solve
  int ntiles;      // Hartley tiles of this solve (same for every axis)
  int nb_dht;      // Hartley blocks of this solve: kTilesPerBlock tiles each
  int nb_vec;      // vector-kernel blocks of this solve
  int pstride;     // partials row stride
  double *x;       // caller's psi (FP64 iterate)
  float *r, *p, *q, *Y, *d;
  Scalars *st_o;   // FP64 refinement scalars
  Scalars *st_i;   // FP32 inner PCG scalars
  double *partials;
  SpectralDev sp;  // FP32 tables of this N
};

__device__ __forceinline__ int find_solve(const int *__restrict__ pre, int count, int b) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void kb_scalars_reset(BSolve *S, int count, double tolrel2, int max_iter, int *iters_total) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  Scalars z;
  memset(&z, 0, sizeof(z));
  z.tolrel2 = tolrel2;
  z.max_iter = max_iter;
  *S[s].st_o = z;
  iters_total[s] = 0;
}

// WHICH 0: outer FP64 residual r32 = b - A x (FIN_RESID on st_o), one node
// row per thread (FP64-ALU-bound);
// WHICH 1: inner FP32 q = A p (FIN_ALPHA on st_i): the shared-memory-staged
// operator (stencil_staged_run) on 32 x 32 tiles where N % 32 == 0, else one
// row per thread.
template <int WHICH, bool GEN>
__global__ void __launch_bounds__(kThreads, WHICH == 1 ? 3 : 1) kb_stencil(const BSolve *__restrict__ S, const int *__restrict__ pre,
                                                       int count) {
  using Ti = typename std::conditional<WHICH == 0, double, float>::type;
  const int s = find_solve(pre, count, blockIdx.x);
  const BSolve &B = S[s];
  Scalars *st = (WHICH == 0) ? B.st_o : B.st_i;
  if (*(volatile int *)&st->done) return;
  // dynamic shared memory: WHICH 1: the staged ring (kStages * kSlot floats),
  // then the pattern tables; WHICH 0: the tables (tab_bytes of the batch's
  // largest layer count)
  extern __shared__ __align__(16) float dsm_b[];
  float *ring = dsm_b;
  Ti(*tab)[kTabStride] = reinterpret_cast<Ti(*)[kTabStride]>(dsm_b + (WHICH == 1 ? kStages * kSlot : 0));
  __shared__ short cellof[kMaxN];
  const int tid = threadIdx.x + 32 * threadIdx.y;
  if constexpr (WHICH == 1) {
    if (B.in_staged) {
      const int N = B.c.N, nbx = N / 32, ntl = nbx * nbx;
      const int lb = blockIdx.x - pre[s];
      const int tile = lb % ntl, zb = lb / ntl;
      const int z0 = zb * B.zc_in, z1 = min(z0 + B.zc_in, N);
      Accum<float> acc;
      stencil_staged_run<GEN>(B.c, B.p, B.q, tab, cellof, ring, (tile / nbx) * 32, (tile % nbx) * 32, z0, z1, acc);
      FF v[2] = {acc.part(), FF{0.f, 0.f}};
      double out[2];
      if (reduce_last_block_ex<2>(v, B.partials, B.pstride, &st->ticket, B.nb_in, lb, out)) {
        if (tid == 0) finalize_scalars(st, FIN_ALPHA, out, 2);
      }
      return;
    }
  }
  build_pattern_table<Ti>(tab, B.c, tid);
  build_cellof(cellof, B.c.N, B.c.n, tid);
  __syncthreads();
  const int N = B.c.N;
  const int lb = blockIdx.x - pre[s];
  const int nbx = (N + 31) / 32, nby = (N + 7) / 8;
  const int bx = lb % nbx, by = (lb / nbx) % nby, bz = lb / (nbx * nby);
  const int j3 = bx * 32 + threadIdx.x, j2 = by * 8 + threadIdx.y;
  const int z0 = bz * B.zc, z1 = min(z0 + B.zc, N);
  Accum<Ti> acc0, acc1;
  if (j3 < N && j2 < N) {
    if constexpr (WHICH == 0)
      stencil_rows<double, float, ST_RESID, 1, GEN>(B.c, B.dir, B.x, B.r, tab, cellof, j3, j2, z0, z1, acc0, acc1);
    else
      stencil_rows<float, float, ST_MATVEC, 1, GEN>(B.c, 0, B.p, B.q, tab, cellof, j3, j2, z0, z1, acc0, acc1);
  }
  typename Accum<Ti>::Part v[2] = {acc0.part(), acc1.part()};
  double out[2];
  if (reduce_last_block_ex<2>(v, B.partials, B.pstride, &st->ticket, WHICH == 1 ? B.nb_in : B.nb_st, lb, out)) {
    if (tid == 0) finalize_scalars(st, WHICH == 0 ? FIN_RESID : FIN_ALPHA, out, 2);
  }
}

// Two-stage tile (see dht_core.cuh) of plan R0 x R1 with P pencils for this
// block's solve.
template <int R0, int R1, int P, int AXIS, int LOADM, int STOREM, bool SCALE>
__device__ __forceinline__ void kb_tile(const BSolve &B, const DhtTile<float> &t, int tile, float2 *sm,
                                        const float2 *tw, float *vtab, Accum<float> &acc) {
  if constexpr (AXIS == 3) {
    __syncthreads();  // twiddles loaded; the previous tile's combine is done with sm
    const size_t row0 = (size_t)tile * 2 * P;
    x3_stage1<float, float2, R0, R1, P, LOADM>(t, row0, sm, acc);
    x3_stage2<float, float2, R0, R1, P>(sm, tw);
    x3_combine<float, float2, R0 * R1, P, STOREM>(t, row0, sm);
  } else if constexpr (SCALE) {
    if (B.sp.rank == 0)
      dht_tile_s2<float, AXIS, R0, R1, P, true, 0>(B.sp, t, tile, sm, tw, vtab, acc);
    else
      dht_tile_s2<float, AXIS, R0, R1, P, true, -1>(B.sp, t, tile, sm, tw, vtab, acc);
  } else {
    dht_tile_s2<float, AXIS, R0, R1, P, false, -1>(B.sp, t, tile, sm, tw, vtab, acc);
  }
}

template <int R0, int R1, int AXIS, int LOADM, int STOREM, bool SCALE>
__device__ __forceinline__ bool kb_tile_p(const BSolve &B, const DhtTile<float> &t, int tile, float2 *sm,
                                          const float2 *tw, float *vtab, Accum<float> &acc) {
  if constexpr ((R0 * R1) % 16 == 0) {
    if (B.logP == 3) {
      kb_tile<R0, R1, 8, AXIS, LOADM, STOREM, SCALE>(B, t, tile, sm, tw, vtab, acc);
      return true;
    }
  }
  if constexpr ((R0 * R1) % 32 == 0) {
    if (B.logP == 4) {
      kb_tile<R0, R1, 16, AXIS, LOADM, STOREM, SCALE>(B, t, tile, sm, tw, vtab, acc);
      return true;
    }
  }
  return false;
}

// The two-stage tile where the solve's N and P have a plan; false otherwise
// (the caller then takes the generic tile). Block-uniform branch.
template <int AXIS, int LOADM, int STOREM, bool SCALE>
__device__ __forceinline__ bool kb_fast_tile(const BSolve &B, const DhtTile<float> &t, int tile, float2 *sm,
                                             const float2 *tw, float *vtab, Accum<float> &acc) {
  switch (B.c.N) {
    case 32: return kb_tile_p<8, 4, AXIS, LOADM, STOREM, SCALE>(B, t, tile, sm, tw, vtab, acc);
    case 48: return kb_tile_p<16, 3, AXIS, LOADM, STOREM, SCALE>(B, t, tile, sm, tw, vtab, acc);
    case 64: return kb_tile_p<8, 8, AXIS, LOADM, STOREM, SCALE>(B, t, tile, sm, tw, vtab, acc);
    case 96: return kb_tile_p<16, 6, AXIS, LOADM, STOREM, SCALE>(B, t, tile, sm, tw, vtab, acc);
    case 128: return kb_tile_p<16, 8, AXIS, LOADM, STOREM, SCALE>(B, t, tile, sm, tw, vtab, acc);
    default: return false;
  }
}

// Inner passes on the FP32 fields of every active solve. A block takes
// kTilesPerBlock consecutive tiles of its solve, so that its fixed start-up
// (finding the solve, its descriptor and stop flag, the twiddles) is paid
// once per several tiles. The 64-register cap lets 4 blocks per SM stay
// resident where shared memory allows (a tile of N = 96, 16 pencils, takes
// 27 KB); only pass C, whose per-N variants are all inlined here, spills.
constexpr int kTilesPerBlock = 4;

template <int AXIS, int LOADM, int STOREM, bool SCALE>
__global__ void __launch_bounds__(kThreads, 4) kb_dht(const BSolve *__restrict__ S, const int *__restrict__ pre,
                                                      int count, int first) {
  using C = float2;
  const int s = find_solve(pre, count, blockIdx.x);
  const BSolve &B = S[s];
  Scalars *st = B.st_i;
  if (*(volatile int *)&st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = B.c.N;
  const int P = 1 << B.logP;
  C *buf0 = reinterpret_cast<C *>(smem_raw);
  C *buf1 = buf0 + N * (P + 1);
  C *tw = buf1 + N * (P + 1);
  float *vtab = reinterpret_cast<float *>(tw + N);
  const C *twg = reinterpret_cast<const C *>(B.sp.tw);
  for (int m = threadIdx.x; m < N; m += kThreads) tw[m] = twg[m];
  DhtTile<float> t;
  const bool pass_a = (AXIS == 3 && STOREM == SO_PLAIN);
  const bool pass_e = (AXIS == 3 && STOREM == SO_PCG);
  t.in = pass_a ? B.r : B.Y;
  t.out = pass_e ? nullptr : B.Y;
  t.r = B.r;
  t.q = B.q;
  t.p = B.p;
  t.x = B.d;
  t.alpha = (float)st->alpha;
  t.beta = (float)st->beta;
  t.first = first;
  t.logP = B.logP;
  const int lb = blockIdx.x - pre[s];
  const int t1 = min(B.ntiles, (lb + 1) * kTilesPerBlock);
  Accum<float> acc;
  // the two-stage tiles use buf0 (and, for x3, part of buf1) as their shared
  // tile; the twiddles and column factors stay where they were loaded; every
  // tile starts with a barrier, so consecutive tiles may reuse the buffers
  for (int tile = lb * kTilesPerBlock; tile < t1; ++tile) {
    if (!kb_fast_tile<AXIS, LOADM, STOREM, SCALE>(B, t, tile, buf0, tw, vtab, acc))
      dht_tile<float, AXIS, LOADM, STOREM, SCALE>(B.sp, t, tile, buf0, buf1, tw, vtab, acc);
  }
  if (LOADM == LD_RESID || SCALE) {
    FF v[1] = {acc.part()};
    double out[1];
    if (reduce_last_block_ex<1>(v, B.partials, B.pstride, &st->ticket, B.nb_dht, lb, out)) {
      if (threadIdx.x == 0) {
        int op = FIN_NONE;
        if (LOADM == LD_RESID) op = first ? FIN_NONE : FIN_RR_ITER;
        if (SCALE) op = first ? FIN_RZ_FIRST : FIN_RZ_BETA;
        finalize_scalars(st, op, out, 1);
      }
    }
  }
}

// Active (not done) solves of the batch -> *out (one block, fixed order).
__global__ void kb_count(const BSolve *__restrict__ S, int count, int which, int *out) {
  __shared__ int sh[kThreads / 32];
  int c = 0;
  for (int s = threadIdx.x; s < count; s += kThreads) {
    const Scalars *st = which == 0 ? S[s].st_o : S[s].st_i;
    c += (*(volatile const int *)&st->done) ? 0 : 1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    *out = t;
  }
}

// Inner solve of A d = r for every solve whose outer residual is not yet small.
__global__ void kb_inner_init(BSolve *S, int count, double tol_in, double tol, int max_iter,
                              const int *iters_total) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  const Scalars *o = S[s].st_o;
  Scalars z;
  memset(&z, 0, sizeof(z));
  const int budget = max_iter - iters_total[s];
  // cut the residual by tol_in, or just enough for the outer tolerance (last step)
  const double need = (o->rr_true > 0.0) ? 0.9 * tol * sqrt(o->bb / o->rr_true) : 1.0;
  const double tin = fmax(tol_in, need);
  z.tolrel2 = tin * tin;
  z.max_iter = budget;
  z.bb = o->rr_true;
  z.tol2 = z.tolrel2 * o->rr_true;
  z.done = (o->done || !(o->rr_true > 0.0) || budget <= 0) ? 1 : 0;
  *S[s].st_i = z;
}

// MODE 0: x = 0; 1: d = 0 (active inner); 2: x += d (+ pending alpha p); 3: x -= mean
template <int MODE>
__global__ void __launch_bounds__(kThreads) kb_vec(const BSolve *__restrict__ S, const int *__restrict__ pre,
                                                   int count) {
  const int s = find_solve(pre, count, blockIdx.x);
  const BSolve &B = S[s];
  const long long n3 = (long long)B.c.N * B.c.N * B.c.N;
  const int lb = blockIdx.x - pre[s];
  if (MODE == 1 && *(volatile int *)&B.st_i->done) return;
  if (MODE == 2 && *(volatile int *)&B.st_o->done) return;
  const float alpha = (float)B.st_i->alpha;
  const int pend = B.st_i->x_pending;
  const double mean = B.st_o->mean;
  for (long long i = (long long)lb * kThreads + threadIdx.x; i < n3; i += (long long)B.nb_vec * kThreads) {
    if (MODE == 0) B.x[i] = 0.0;
    if (MODE == 1) B.d[i] = 0.f;
    if (MODE == 2) {
      float dd = B.d[i];
      if (pend) dd = fmaf(alpha, B.p[i], dd);
      B.x[i] += (double)dd;
    }
    if (MODE == 3) B.x[i] -= mean;
  }
}

// sum(x) per solve -> st_o->mean
__global__ void __launch_bounds__(kThreads) kb_mean(const BSolve *__restrict__ S, const int *__restrict__ pre,
                                                    int count) {
  const int s = find_solve(pre, count, blockIdx.x);
  const BSolve &B = S[s];
  const long long n3 = (long long)B.c.N * B.c.N * B.c.N;
  const int lb = blockIdx.x - pre[s];
  double acc = 0.0;
  for (long long i = (long long)lb * kThreads + threadIdx.x; i < n3; i += (long long)B.nb_vec * kThreads) acc += B.x[i];
  double v[1] = {acc}, out[1];
  if (reduce_last_block_ex<1>(v, B.partials, B.pstride, &B.st_o->ticket, B.nb_vec, lb, out)) {
    if (threadIdx.x == 0) B.st_o->mean = out[0] / (double)n3;
  }
}

__global__ void kb_accum_iters(const BSolve *__restrict__ S, int count, int *iters_total) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < count) iters_total[s] += S[s].st_i->iter;
}

}  // namespace sq

using namespace sq;

struct sq_batch {
  int count;
  std::vector<BSolve> hS;
  BSolve *dS = nullptr;
  int *d_pre = nullptr;  // [0..count] stencil, [count+1..] dht, [2count+2..] vec, [3count+3..] inner stencil
  int tot_st = 0, tot_dht = 0, tot_vec = 0, tot_in = 0;
  size_t dht_smem[2] = {0, 0};  // plain passes, pass C
  int layers = 1;               // most threshold layers of the batch's media (pattern tables)
  bool general = false;         // some medium is not the plain checkerboard (see general_media)
  void *d_mem = nullptr;        // fields, scalars, partials
  int *d_iters = nullptr;
  int *d_count = nullptr;
  int *h_count = nullptr;       // pinned
  int *h_iters = nullptr;       // pinned
  Scalars *h_st = nullptr;      // pinned, count
  Scalars *d_sc = nullptr;      // 2 per solve: outer, inner
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cudaEvent_t ev = nullptr;
};

namespace {

// Inner iterations per graph replay (the host polls one replay behind):
// 768 mixed solves measured 4315 / 4449 solves/s with 8 / 4.
constexpr int kChunk = 4;
constexpr size_t kStagedSmem = (size_t)kStages * kSlot * sizeof(float);  // ring of the staged inner operator

#define SQB_CK(call)                        \
  do {                                      \
    if ((call) != cudaSuccess) return SQ_ECUDA; \
  } while (0)

template <int AXIS, int LOADM, int STOREM, bool SCALE>
int launch_kb_dht(sq_batch *b, int first, cudaStream_t s) {
  const size_t smem = b->dht_smem[SCALE ? 1 : 0];
  kb_dht<AXIS, LOADM, STOREM, SCALE><<<b->tot_dht, kThreads, smem, s>>>(b->dS, b->d_pre + b->count + 1, b->count,
                                                                        first);
  return cudaGetLastError() == cudaSuccess ? SQ_OK : SQ_ECUDA;
}

template <int AXIS, int LOADM, int STOREM, bool SCALE>
int set_kb_dht_smem(size_t smem) {
  return cudaFuncSetAttribute(kb_dht<AXIS, LOADM, STOREM, SCALE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem) == cudaSuccess
             ? SQ_OK
             : SQ_ECUDA;
}

int precond_first_b(sq_batch *b, cudaStream_t s) {
  int st;
  if ((st = launch_kb_dht<3, LD_PLAIN, SO_PLAIN, false>(b, 1, s)) != SQ_OK) return st;
  if ((st = launch_kb_dht<2, LD_PLAIN, SO_PLAIN, false>(b, 1, s)) != SQ_OK) return st;
  if ((st = launch_kb_dht<1, LD_PLAIN, SO_PLAIN, true>(b, 1, s)) != SQ_OK) return st;
  if ((st = launch_kb_dht<2, LD_PLAIN, SO_PLAIN, false>(b, 1, s)) != SQ_OK) return st;
  return launch_kb_dht<3, LD_PLAIN, SO_PCG, false>(b, 1, s);
}

// One inner PCG iteration of every active solve: six launches (each bracketed
// by the kernel-event profile when it is on; outside a capture only).
int iteration_b(sq_batch *b, cudaStream_t s) {
  size_t pi = profile_begin_batch_inner(s);
  if (b->general)
    kb_stencil<1, true><<<b->tot_in, dim3(32, 8, 1), kStagedSmem + tab_bytes<float>(b->layers), s>>>(
        b->dS, b->d_pre + 3 * (b->count + 1), b->count);
  else
    kb_stencil<1, false><<<b->tot_in, dim3(32, 8, 1), kStagedSmem + tab_bytes<float>(1), s>>>(
        b->dS, b->d_pre + 3 * (b->count + 1), b->count);
  profile_end(pi, s);
  if (cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
  int st;
#define SQB_PROF(call)                       \
  pi = profile_begin_batch_inner(s);         \
  st = (call);                               \
  profile_end(pi, s);                        \
  if (st != SQ_OK) return st;
  SQB_PROF((launch_kb_dht<3, LD_RESID, SO_PLAIN, false>(b, 0, s)));
  SQB_PROF((launch_kb_dht<2, LD_PLAIN, SO_PLAIN, false>(b, 0, s)));
  SQB_PROF((launch_kb_dht<1, LD_PLAIN, SO_PLAIN, true>(b, 0, s)));
  SQB_PROF((launch_kb_dht<2, LD_PLAIN, SO_PLAIN, false>(b, 0, s)));
  SQB_PROF((launch_kb_dht<3, LD_PLAIN, SO_PCG, false>(b, 0, s)));
#undef SQB_PROF
  return SQ_OK;
}

int capture_graph(sq_batch *b, cudaStream_t s) {
  if (b->exec) return SQ_OK;
  // A private stream for the capture keeps the caller's stream untouched.
  cudaStream_t cs;
  SQB_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int st = SQ_OK;
  profile_pause(true);  // no event records inside the capture
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = SQ_ECUDA;
  for (int i = 0; st == SQ_OK && i < kChunk; ++i) st = iteration_b(b, cs);
  if (st == SQ_OK) {
    kb_count<<<1, kThreads, 0, cs>>>(b->dS, b->count, 1, b->d_count);
    if (cudaGetLastError() != cudaSuccess) st = SQ_ECUDA;
  }
  if (st == SQ_OK &&
      cudaMemcpyAsync(b->h_count, b->d_count, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
    st = SQ_ECUDA;
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g) st = SQ_ECUDA;
  if (st == SQ_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) st = SQ_ECUDA;
  b->graph = g;
  profile_pause(false);
  cudaStreamDestroy(cs);
  (void)s;
  return st;
}

int count_active(sq_batch *b, int which, cudaStream_t s, int *out) {
  kb_count<<<1, kThreads, 0, s>>>(b->dS, b->count, which, b->d_count);
  SQB_CK(cudaGetLastError());
  SQB_CK(cudaMemcpyAsync(b->h_count, b->d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
  SQB_CK(cudaStreamSynchronize(s));
  *out = *b->h_count;
  return SQ_OK;
}

bool valid_N_b(int N) {
  if (N < 8 || N > kMaxN || (N & 1)) return false;
  int m = N;
  while (m % 2 == 0) m /= 2;
  if (m % 3 == 0) m /= 3;
  return m == 1;
}

}  // namespace


extern "C" {

int sq_batch_create(int count, const sq_solve_desc *descs, const sq_precond *const *precs,
                    const sq_tile_config *tiles, int ntiles, sq_batch **out) {
  if (!out || count < 1 || !descs || !precs || (ntiles > 0 && !tiles)) return SQ_EINVAL;
  *out = nullptr;
  sq_batch *b = new (std::nothrow) sq_batch();
  if (!b) return SQ_ENOMEM;
  b->count = count;
  b->hS.resize(count);
  std::vector<int> pre((size_t)4 * (count + 1), 0);
  size_t field_floats = 0;
  int maxN = 0, maxR = 0, maxP = 1;
  for (int k = 0; k < count; ++k) {
    CellsDev cv;
    SpectralDev sp;
    int pN = 0;
    if (!descs[k].coeffs || !descs[k].psi || descs[k].dir < 0 || descs[k].dir > 2 || !precs[k] ||
        coeffs_view(descs[k].coeffs, &cv) != SQ_OK || precond_spec32(precs[k], &sp, &pN) != SQ_OK || pN != cv.N ||
        !valid_N_b(cv.N)) {
      delete b;
      return SQ_EINVAL;
    }
    BSolve &B = b->hS[k];
    memset(&B, 0, sizeof(B));
    B.c = cv;
    B.dir = descs[k].dir;
    B.x = descs[k].psi;
    B.sp = sp;
    B.sp.gtab = nullptr;  // the batch evaluates the multiplier on the fly (its shared memory has no table slot)
    const int N = cv.N;
    int P = dht_tile_pencils(N, 4);
    int zc = std::max(2, N / 4);
    for (int t = 0; t < ntiles; ++t)
      if (tiles[t].N == N) {
        if (tiles[t].dht_pencils > 0) P = tiles[t].dht_pencils;
        if (tiles[t].stencil_planes > 0) zc = tiles[t].stencil_planes;
      }
    if (P < 1 || (P & (P - 1)) || N % (2 * P) != 0 || dht_smem_bytes_t<float>(N, P, sp.rank) > 200 * 1024 || zc < 1 ||
        zc > N) {
      delete b;
      return SQ_EINVAL;
    }
    int logP = 0;
    while ((1 << logP) < P) ++logP;
    B.logP = logP;
    B.zc = zc;
    B.nb_st = ((N + 31) / 32) * ((N + 7) / 8) * ((N + zc - 1) / zc);
    B.in_staged = (N % 32 == 0) ? 1 : 0;
    if (B.in_staged) {
      B.zc_in = std::min(N, 16);
      B.nb_in = (N / 32) * (N / 32) * ((N + B.zc_in - 1) / B.zc_in);
    } else {
      B.zc_in = zc;
      B.nb_in = B.nb_st;
    }
    B.ntiles = N * N / (2 * P);
    B.nb_dht = (B.ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
    const long long n3 = (long long)N * N * N;
    B.nb_vec = (int)std::max(1LL, std::min(4096LL, n3 / (kThreads * 8)));
    B.pstride = std::max(std::max(B.nb_st, B.nb_in), std::max(B.nb_dht, B.nb_vec));
    pre[k + 1] = pre[k] + B.nb_st;
    pre[(count + 1) + k + 1] = pre[(count + 1) + k] + B.nb_dht;
    pre[2 * (count + 1) + k + 1] = pre[2 * (count + 1) + k] + B.nb_vec;
    pre[3 * (count + 1) + k + 1] = pre[3 * (count + 1) + k] + B.nb_in;
    field_floats += 5 * (size_t)n3;
    maxN = std::max(maxN, N);
    b->layers = std::max(b->layers, B.c.layers);
    b->general = b->general || general_media(B.c);
    maxR = std::max(maxR, sp.rank);
    maxP = std::max(maxP, P);
    b->dht_smem[0] = std::max(b->dht_smem[0], dht_smem_bytes_t<float>(N, P, 0));
    b->dht_smem[1] = std::max(b->dht_smem[1], dht_smem_bytes_t<float>(N, P, sp.rank));
  }
  b->tot_st = pre[count];
  b->tot_dht = pre[(count + 1) + count];
  b->tot_vec = pre[2 * (count + 1) + count];
  b->tot_in = pre[3 * (count + 1) + count];
  // one allocation: FP32 fields, scalars (2 per solve), partials
  size_t partials = 0;
  for (auto &B : b->hS) partials += (size_t)2 * B.pstride;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t bytes_fields = al(field_floats * sizeof(float));
  const size_t bytes_scal = al((size_t)2 * count * sizeof(Scalars));
  const size_t bytes_part = al(partials * sizeof(double));
  bool ok = cudaMalloc(&b->d_mem, bytes_fields + bytes_scal + bytes_part) == cudaSuccess;
  ok = ok && cudaMalloc(&b->dS, sizeof(BSolve) * count) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_pre, sizeof(int) * pre.size()) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_iters, sizeof(int) * count) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_count, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_count, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_iters, sizeof(int) * count) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_st, 2 * sizeof(Scalars) * count) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    sq_batch_destroy(b);
    return SQ_ENOMEM;
  }
  char *base = static_cast<char *>(b->d_mem);
  float *fp = reinterpret_cast<float *>(base);
  Scalars *sc = reinterpret_cast<Scalars *>(base + bytes_fields);
  double *pp = reinterpret_cast<double *>(base + bytes_fields + bytes_scal);
  b->d_sc = sc;
  for (int k = 0; k < count; ++k) {
    BSolve &B = b->hS[k];
    const size_t n3 = (size_t)B.c.N * B.c.N * B.c.N;
    B.r = fp;
    B.p = fp + n3;
    B.q = fp + 2 * n3;
    B.Y = fp + 3 * n3;
    B.d = fp + 4 * n3;
    fp += 5 * n3;
    B.st_o = sc + 2 * k;
    B.st_i = sc + 2 * k + 1;
    B.partials = pp;
    pp += 2 * (size_t)B.pstride;
  }
  ok = cudaMemcpy(b->dS, b->hS.data(), sizeof(BSolve) * count, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(b->d_pre, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemset(sc, 0, bytes_scal) == cudaSuccess;
  ok = ok && allow_dynamic_smem(b->general ? (const void *)kb_stencil<1, true> : (const void *)kb_stencil<1, false>,
                                kStagedSmem + tab_bytes<float>(b->layers)) == cudaSuccess;
  ok = ok && allow_dynamic_smem(b->general ? (const void *)kb_stencil<0, true> : (const void *)kb_stencil<0, false>,
                                tab_bytes<double>(b->layers)) == cudaSuccess;
  ok = ok && set_kb_dht_smem<3, LD_PLAIN, SO_PLAIN, false>(b->dht_smem[0]) == SQ_OK;
  ok = ok && set_kb_dht_smem<3, LD_RESID, SO_PLAIN, false>(b->dht_smem[0]) == SQ_OK;
  ok = ok && set_kb_dht_smem<2, LD_PLAIN, SO_PLAIN, false>(b->dht_smem[0]) == SQ_OK;
  ok = ok && set_kb_dht_smem<1, LD_PLAIN, SO_PLAIN, true>(b->dht_smem[1]) == SQ_OK;
  ok = ok && set_kb_dht_smem<3, LD_PLAIN, SO_PCG, false>(b->dht_smem[0]) == SQ_OK;
  if (!ok) {
    sq_batch_destroy(b);
    return SQ_ECUDA;
  }
  (void)maxN;
  (void)maxR;
  (void)maxP;
  *out = b;
  return SQ_OK;
}

void sq_batch_destroy(sq_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_mem) cudaFree(b->d_mem);
  if (b->dS) cudaFree(b->dS);
  if (b->d_pre) cudaFree(b->d_pre);
  if (b->d_iters) cudaFree(b->d_iters);
  if (b->d_count) cudaFree(b->d_count);
  if (b->h_count) cudaFreeHost(b->h_count);
  if (b->h_iters) cudaFreeHost(b->h_iters);
  if (b->h_st) cudaFreeHost(b->h_st);
  if (b->ev) cudaEventDestroy(b->ev);
  delete b;
}

int sq_pcg_solve_batched(sq_batch *b, double tol, int max_iter, sq_solve_info *infos, sq_stream_t stream) {
  if (!b || !(tol > 0.0) || max_iter < 1) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int count = b->count;
  const int *pre_vec = b->d_pre + 2 * (count + 1);
  const double tol_in = inner_tol();
  int st = capture_graph(b, s);
  if (st != SQ_OK) return st;
  const int tb = (count + 127) / 128;
  kb_scalars_reset<<<tb, 128, 0, s>>>(b->dS, count, tol * tol, max_iter, b->d_iters);
  kb_vec<0><<<b->tot_vec, kThreads, 0, s>>>(b->dS, pre_vec, count);
  SQB_CK(cudaGetLastError());
  int outer = 0;
  for (; outer < 30; ++outer) {
    if (b->general)
      kb_stencil<0, true><<<b->tot_st, dim3(32, 8, 1), tab_bytes<double>(b->layers), s>>>(b->dS, b->d_pre, count);
    else
      kb_stencil<0, false><<<b->tot_st, dim3(32, 8, 1), tab_bytes<double>(1), s>>>(b->dS, b->d_pre, count);
    SQB_CK(cudaGetLastError());
    int active = 0;
    if ((st = count_active(b, 0, s, &active)) != SQ_OK) return st;
    if (active == 0) break;
    kb_inner_init<<<tb, 128, 0, s>>>(b->dS, count, tol_in, tol, max_iter, b->d_iters);
    kb_vec<1><<<b->tot_vec, kThreads, 0, s>>>(b->dS, pre_vec, count);
    SQB_CK(cudaGetLastError());
    if ((st = precond_first_b(b, s)) != SQ_OK) return st;
    // inner iterations: graph chunks, polled one chunk behind (with the
    // profile on: the same launches one by one, each and the loop timed)
    int launched = 0;
    bool pending = false;
    const size_t ploop = profile_begin_batch_loop(s);
    while (launched < max_iter) {
      if (profile_enabled()) {  // the graph's contents, launched one by one and timed by the profile
        for (int i = 0; i < kChunk; ++i)
          if ((st = iteration_b(b, s)) != SQ_OK) return st;
        kb_count<<<1, kThreads, 0, s>>>(b->dS, b->count, 1, b->d_count);
        SQB_CK(cudaGetLastError());
        SQB_CK(cudaMemcpyAsync(b->h_count, b->d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
      } else {
        SQB_CK(cudaGraphLaunch(b->exec, s));
      }
      launched += kChunk;
      if (pending) {
        SQB_CK(cudaEventSynchronize(b->ev));
        if (*b->h_count == 0) break;
      }
      SQB_CK(cudaEventRecord(b->ev, s));
      pending = true;
    }
    profile_end(ploop, s);
    kb_vec<2><<<b->tot_vec, kThreads, 0, s>>>(b->dS, pre_vec, count);
    kb_accum_iters<<<tb, 128, 0, s>>>(b->dS, count, b->d_iters);
    SQB_CK(cudaGetLastError());
  }
  kb_mean<<<b->tot_vec, kThreads, 0, s>>>(b->dS, pre_vec, count);
  kb_vec<3><<<b->tot_vec, kThreads, 0, s>>>(b->dS, pre_vec, count);
  SQB_CK(cudaGetLastError());
  SQB_CK(cudaMemcpyAsync(b->h_st, b->d_sc, 2 * sizeof(Scalars) * count, cudaMemcpyDeviceToHost, s));
  SQB_CK(cudaMemcpyAsync(b->h_iters, b->d_iters, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
  SQB_CK(cudaStreamSynchronize(s));
  int status = SQ_OK;
  for (int k = 0; k < count; ++k) {
    const Scalars &h = b->h_st[2 * k];  // outer scalars of solve k
    sq_solve_info tmp;
    sq_solve_info &inf = infos ? infos[k] : tmp;
    inf.iters = b->h_iters[k];
    inf.outer_steps = outer;
    inf.used_guess = 0;
    inf.relres = 0.0;
    inf.relres_true = (h.bb > 0.0) ? std::sqrt(h.rr_true / h.bb) : 0.0;
    inf.status = (h.bb == 0.0 || inf.relres_true <= tol) ? SQ_OK : SQ_ENOCONV;
    if (inf.status != SQ_OK) status = SQ_ENOCONV;
  }
  return status;
}

}  // extern "C"
