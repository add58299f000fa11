// Cell generation, the matrix-free stiffness operator, right-hand sides,
// homogenized matrix and small vector kernels.
//
// Operator (Sec. 3.2-3.3, Eqs. 9 and 18, read as the lumped form
// A = sum_d D_d^T diag(a_d) D_d): for node j,
//   (A x)(j) = sum_d a_d(j) (x(j) - x(j+e_d)) + a_d(j-e_d) (x(j) - x(j-e_d)),
// where a_d(j) is the mean of the four grid voxels around the edge j -> j+e_d
// (the Kronecker-sum weights Ihat = diag{1/2,1,..,1,1/2} of Sec. 3.3 summed over
// the cells sharing that edge: 1, 1/2 or 1/4 per cell). Every voxel takes the
// value of its cell, so the eight voxels around a node -- one bit each, read
// from the L^3 phase array -- fix all six edge coefficients of that node. A
// 256-entry table per block maps this 8-bit pattern to the six coefficients
// and the diagonal; no N^3 coefficient field exists. Multi-level media (K
// coefficient levels) add one table per extra threshold layer; the node's
// coefficients are the sum of its layers' rows (see CellsDev).
//
// RHS (Eq. 8 in grid units): b_dir(j) = a_dir(j) - a_dir(j - e_dir).
#include <mutex>

#include "stencil_core.cuh"

namespace sq {

// --------------------------------------------------------------- cell phases
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number i of the stream
// seeded with `seed` is mix(seed + (i+1) * golden_gamma).
__device__ __forceinline__ uint64_t splitmix64_output(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Level of cell i = the number of thresholds t1 >= t2 >= t3 above the top 53
// bits u of its output (two-level media: t2 = t3 = 0, level = [u < t1]).
__global__ void k_coeff_gen(uint8_t *__restrict__ phase, int ncell, uint64_t seed, uint64_t t1, uint64_t t2,
                            uint64_t t3) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncell) {
    const uint64_t u = splitmix64_output(seed, (uint64_t)i) >> 11;
    phase[i] = (uint8_t)((u < t1 ? 1 : 0) + (u < t2 ? 1 : 0) + (u < t3 ? 1 : 0));
  }
}

cudaError_t launch_coeff_gen_cells(uint8_t *phase, int ncell, uint64_t seed, const uint64_t *thr, cudaStream_t s) {
  k_coeff_gen<<<(ncell + 255) / 256, 256, 0, s>>>(phase, ncell, seed, thr[0], thr[1], thr[2]);
  return cudaGetLastError();
}

cudaError_t launch_coeff_gen(uint8_t *phase, int L, uint64_t seed, const uint64_t *thr, cudaStream_t s) {
  return launch_coeff_gen_cells(phase, L * L * L, seed, thr, s);
}

// Work item = a tile of 32 node columns (j3) x 8 RPT node rows (j2) times a
// chunk of zc planes along j1; items are numbered with j3 tiles fastest, then
// j2 tiles, then chunks, so concurrently running blocks share their halo rows
// in L2. The grid holds as many blocks as fit on the GPU at once and each
// block loops over items: the tables are built and the block's partial sums
// reduced once per block, not once per item. RPT > 1 (FP32, N divisible by
// RPT) amortises the per-plane index and coefficient work over RPT rows at
// the cost of registers (RPT 4: ~114, two blocks per SM; RPT 2: ~64, four);
// FP64 (ALU-bound) keeps one row per thread.
template <typename Ti, typename To, int MODE, int RPT, bool GEN>
__global__ void __launch_bounds__(kThreads) k_stencil(CellsDev c, int dir, const Ti *__restrict__ x,
                                                      To *__restrict__ y, RedBuf rb, int fin, int check_done,
                                                      int zc, int nitems) {
  if (check_done && *(volatile int *)&rb.st->done) return;
  extern __shared__ __align__(16) unsigned char dsm[];  // pattern tables, tab_bytes<Ti>(c.layers)
  Ti(*tab)[kTabStride] = reinterpret_cast<Ti(*)[kTabStride]>(dsm);
  __shared__ short cellof[kMaxN];
  const int tid = threadIdx.x + 32 * threadIdx.y;
  build_pattern_table<Ti>(tab, c, tid);
  build_cellof(cellof, c.N, c.n, tid);
  __syncthreads();
  const int N = c.N;
  const int nbx = (N + 31) / 32, nby = (N + 8 * RPT - 1) / (8 * RPT);
  Accum<Ti> acc0, acc1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int bx = it % nbx, rest = it / nbx;
    const int by = rest % nby, bz = rest / nby;
    const int j3 = bx * 32 + threadIdx.x;
    const int j2b = (by * 8 + threadIdx.y) * RPT;
    const int z0 = bz * zc;
    const int z1 = min(z0 + zc, N);
    if (j3 < N && j2b < N)
      stencil_rows<Ti, To, MODE, RPT, GEN>(c, dir, x, y, tab, cellof, j3, j2b, z0, z1, acc0, acc1);
  }
  typename Accum<Ti>::Part v[2] = {acc0.part(), acc1.part()};
  double s[2];
  if (reduce_last_block<2>(v, rb.partials, &rb.st->ticket, s)) {
    if (tid == 0) finalize_scalars(rb.st, fin, s, 2);
  }
}

// Raises a kernel's dynamic shared-memory limit to `smem` bytes where that is
// above the default 48 KB (once per kernel and device; guarded for
// concurrent host threads).
cudaError_t allow_dynamic_smem(const void *kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  struct Entry {
    const void *k;
    int dev;
    size_t smem;
  };
  static Entry done[64];
  static int used = 0;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i)
    if (done[i].k == kern && done[i].dev == dev && done[i].smem >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && used < 64) done[used++] = Entry{kern, dev, smem};
  return e;
}

// Blocks that fit on the device at once for one kernel (cached per kernel and
// device; the cache is guarded for concurrent host threads); 0 on error.
static int resident_blocks(const void *kern, int threads, size_t smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  struct Entry {
    const void *k;
    int dev;
    size_t smem;
    int blocks;
  };
  static Entry cache[64];
  static int used = 0;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; ++i)
      if (cache[i].k == kern && cache[i].dev == dev && cache[i].smem == smem) return cache[i].blocks;
  }
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int blocks = per_sm * sms;
  std::lock_guard<std::mutex> lock(mu);
  if (used < 64) cache[used++] = Entry{kern, dev, smem, blocks};
  return blocks;
}

static int g_planes_override[kMaxN + 1] = {0};  // FP32 operator planes per work item, per N (0 = default)

// Staged FP32 operator over one (tile, plane run) per block; see stencil_staged_run.
template <bool GEN>
__global__ void __launch_bounds__(kThreads, 3) k_stencil_staged(CellsDev c, const float *__restrict__ x,
                                                             float *__restrict__ y, RedBuf rb, int fin,
                                                             int check_done, int zc, int ntiles) {
  if (check_done && *(volatile int *)&rb.st->done) return;
  extern __shared__ __align__(16) float ring[];  // kStages slots of kSlot floats, then the pattern tables
  float(*tab)[kTabStride] = reinterpret_cast<float(*)[kTabStride]>(ring + kStages * kSlot);
  __shared__ short cellof[kMaxN];
  const int N = c.N;
  const int nbx = N / 32;
  const int tile = blockIdx.x % ntiles, zb = blockIdx.x / ntiles;
  const int z0 = zb * zc, z1 = min(z0 + zc, N);
  Accum<float> acc;
  stencil_staged_run<GEN>(c, x, y, tab, cellof, ring, (tile / nbx) * 32, (tile % nbx) * 32, z0, z1, acc);
  FF v[2] = {acc.part(), FF{0.f, 0.f}};
  double sres[2];
  if (reduce_last_block<2>(v, rb.partials, &rb.st->ticket, sres)) {
    if (threadIdx.x + 32 * threadIdx.y == 0) finalize_scalars(rb.st, fin, sres, 2);
  }
}

template <bool GEN>
static cudaError_t launch_stencil_staged(const CellsDev &c, const float *x, float *y, RedBuf rb, int fin,
                                         bool check_done, cudaStream_t s) {
  const int N = c.N;
  const size_t smem = (size_t)kStages * kSlot * sizeof(float) + tab_bytes<float>(c.layers);
  auto kern = k_stencil_staged<GEN>;
  const cudaError_t e = allow_dynamic_smem((const void *)kern, smem);
  if (e != cudaSuccess) return e;
  const int ntiles = (N / 32) * (N / 32);
  const int resident = resident_blocks((const void *)kern, kThreads, smem);
  if (resident <= 0) return cudaErrorInvalidConfiguration;
  int nz = resident / ntiles;
  if (nz > N / 4) nz = N / 4;  // at least 4 planes per block
  if (nz < 1) nz = 1;
  int zc = (N + nz - 1) / nz;  // one wave of resident blocks
  if (g_planes_override[N] >= 4) zc = g_planes_override[N];  // a tuned plane run (longer runs, fewer blocks)
  nz = (N + zc - 1) / zc;
  const long long grid = (long long)ntiles * nz;
  if (grid > kMaxPartials) return cudaErrorInvalidConfiguration;
  kern<<<(int)grid, dim3(32, 8, 1), smem, s>>>(c, x, y, rb, fin, check_done ? 1 : 0, zc, ntiles);
  return cudaGetLastError();
}

static int g_stencil_rows = 0;  // FP32 operator: 0 automatic, 1 / 2 / 4 rows per thread, 8 staged

static int g_rows_override[kMaxN + 1] = {0};

static bool valid_rows(int rpt) { return rpt == 0 || rpt == 1 || rpt == 2 || rpt == 4 || rpt == 8; }

int set_stencil_rows(int rpt) {
  if (!valid_rows(rpt)) return 1;
  g_stencil_rows = rpt;
  return 0;
}

int set_stencil_rows_override(int N, int rpt) {
  if (N < 8 || N > kMaxN || !valid_rows(rpt)) return 1;
  g_rows_override[N] = rpt;
  return 0;
}

int set_stencil_planes_override(int N, int zc) {
  if (N < 8 || N > kMaxN) return 1;
  if (zc != 0 && (zc < 1 || zc > N)) return 1;
  g_planes_override[N] = zc;
  return 0;
}

static int stencil_zc(int N, int rpt) {
  if (N >= 8 && N <= kMaxN && g_planes_override[N]) return g_planes_override[N];
  // about 4 K items of 4 to 16 planes
  const long long tiles = (long long)((N + 31) / 32) * ((N + 8 * rpt - 1) / (8 * rpt));
  int zc = (int)((tiles * N + 4095) / 4096);
  if (zc < 4) zc = 4;
  if (zc > 16) zc = 16;
  if (zc > N) zc = N;
  return zc;
}

template <typename Ti, typename To, int MODE, int RPT, bool GEN = false>
static cudaError_t launch_stencil_mode(const CellsDev &c, int dir, const Ti *x, To *y, RedBuf rb, int fin,
                                       bool check_done, cudaStream_t s) {
  const int N = c.N;
  const int zc = stencil_zc(N, RPT);
  const long long items =
      (long long)((N + 31) / 32) * ((N + 8 * RPT - 1) / (8 * RPT)) * ((N + zc - 1) / zc);
  auto kern = k_stencil<Ti, To, MODE, RPT, GEN>;
  const size_t smem = tab_bytes<Ti>(c.layers);
  const cudaError_t e = allow_dynamic_smem((const void *)kern, smem);
  if (e != cudaSuccess) return e;
  long long grid = resident_blocks((const void *)kern, kThreads, smem);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  if (grid > items) grid = items;
  if (grid > kMaxPartials) grid = kMaxPartials;
  kern<<<(int)grid, dim3(32, 8, 1), smem, s>>>(c, dir, x, y, rb, fin, check_done ? 1 : 0, zc, (int)items);
  return cudaGetLastError();
}

// Media other than the plain checkerboard (several levels or sub-cell
// inclusions) take the kernels compiled for them: the staged FP32 operator
// where it applies, else one row per thread.
template <typename Ti, typename To, int MODE>
static cudaError_t launch_stencil_rows(const CellsDev &c, int dir, const Ti *x, To *y, RedBuf rb, int fin,
                                       bool check_done, cudaStream_t s) {
  if (general_media(c)) {
    if constexpr (sizeof(Ti) == 4 && MODE == ST_MATVEC && sizeof(To) == 4) {
      if (c.N % 32 == 0 && ((uintptr_t)x & 15) == 0) return launch_stencil_staged<true>(c, x, y, rb, fin, check_done, s);
    }
    return launch_stencil_mode<Ti, To, MODE, 1, true>(c, dir, x, y, rb, fin, check_done, s);
  }
  if constexpr (sizeof(Ti) == 4) {
    const int per_n = (c.N >= 8 && c.N <= kMaxN) ? g_rows_override[c.N] : 0;
    const int want = per_n ? per_n : (g_stencil_rows ? g_stencil_rows : 8);
    if constexpr (MODE == ST_MATVEC && sizeof(To) == 4) {
      if (want == 8 && c.N % 32 == 0 && ((uintptr_t)x & 15) == 0)
        return launch_stencil_staged<false>(c, x, y, rb, fin, check_done, s);
    }
    if (want >= 4 && c.N % 4 == 0) return launch_stencil_mode<Ti, To, MODE, 4>(c, dir, x, y, rb, fin, check_done, s);
    if (want >= 2 && c.N % 2 == 0) return launch_stencil_mode<Ti, To, MODE, 2>(c, dir, x, y, rb, fin, check_done, s);
  }
  return launch_stencil_mode<Ti, To, MODE, 1>(c, dir, x, y, rb, fin, check_done, s);
}

template <typename Ti, typename To>
cudaError_t launch_stencil(const CellsDev &c, int mode, int dir, const Ti *x, To *y, RedBuf rb, int fin,
                           bool check_done, cudaStream_t s) {
  switch (mode) {
    case ST_MATVEC: return launch_stencil_rows<Ti, To, ST_MATVEC>(c, dir, x, y, rb, fin, check_done, s);
    case ST_RESID: return launch_stencil_rows<Ti, To, ST_RESID>(c, dir, x, y, rb, fin, check_done, s);
    default: return launch_stencil_rows<Ti, To, ST_RHS>(c, dir, x, y, rb, fin, check_done, s);
  }
}

template cudaError_t launch_stencil<double, double>(const CellsDev &, int, int, const double *, double *, RedBuf,
                                                    int, bool, cudaStream_t);
template cudaError_t launch_stencil<float, float>(const CellsDev &, int, int, const float *, float *, RedBuf, int,
                                                  bool, cudaStream_t);
template cudaError_t launch_stencil<double, float>(const CellsDev &, int, int, const double *, float *, RedBuf,
                                                   int, bool, cudaStream_t);

// --------------------------------------------------------- homogenized matrix
// Eq. 21 on the grid: A_ij = delta_ij mean(a_j) + mean(a_j D_j psi_i) (edge
// form, the paper's Eq. 23 after summation by parts) and the energy form
// E_ij = mean(sum_d a_d (delta_id + D_d psi_i)(delta_jd + D_d psi_j)).
// Reduced quantities: 0..8 M[i][j] = sum a_j D_j psi_i, 9..11 sum a_j,
// 12..17 energy sums for (i,j) in (00,01,02,11,12,22).
// ENERGY = false skips the six energy sums (most of the kernel's FP64 work)
// when the caller only wants the edge form.
template <bool ENERGY>
__global__ void __launch_bounds__(kThreads) k_ahom(CellsDev c, const double *__restrict__ p0,
                                                   const double *__restrict__ p1, const double *__restrict__ p2,
                                                   RedBuf rb, int zc) {
  extern __shared__ __align__(16) unsigned char dsm[];  // pattern tables, tab_bytes<double>(c.layers)
  double(*tab)[kTabStride] = reinterpret_cast<double(*)[kTabStride]>(dsm);
  const int tid = threadIdx.x + 32 * threadIdx.y;
  build_pattern_table<double>(tab, c, tid);
  __syncthreads();
  const int N = c.N, n = c.n, L = c.L;
  const size_t NN = (size_t)N * N;
  const int j3 = blockIdx.x * 32 + threadIdx.x;
  const int j2 = blockIdx.y * 8 + threadIdx.y;
  const int z0 = blockIdx.z * zc;
  const int z1 = min(z0 + zc, N);
  double acc[18];
#pragma unroll
  for (int q = 0; q < 18; ++q) acc[q] = 0.0;
  if (j3 < N && j2 < N) {
    const int j3m = (j3 == 0) ? N - 1 : j3 - 1, j3p = (j3 == N - 1) ? 0 : j3 + 1;
    const int j2m = (j2 == 0) ? N - 1 : j2 - 1, j2p = (j2 == N - 1) ? 0 : j2 + 1;
    const int c3a = j3 / n, c3b = j3m / n, c2a = j2 / n, c2b = j2m / n;
    const int LL = L * L;
    const int o00 = c2a * L + c3a, o01 = c2a * L + c3b, o10 = c2b * L + c3a, o11 = c2b * L + c3b;
    // sub-cell inclusions: which of the four in-plane voxels may be high (load4's bit order)
    const bool i2a = in_sub(c, j2 - c2a * n), i2b = in_sub(c, j2m - c2b * n);
    const bool i3a = in_sub(c, j3 - c3a * n), i3b = in_sub(c, j3m - c3b * n);
    const unsigned m23 =
        all_layers((i2a && i3a ? 1u : 0u) | (i2a && i3b ? 2u : 0u) | (i2b && i3a ? 4u : 0u) | (i2b && i3b ? 8u : 0u));
    const double *ps[3] = {p0, p1, p2};
    for (int j1 = z0; j1 < z1; ++j1) {
      const int j1m = (j1 == 0) ? N - 1 : j1 - 1, j1p = (j1 == N - 1) ? 0 : j1 + 1;
      const unsigned pm0 = in_sub(c, j1 - (j1 / n) * n) ? m23 : 0u, pm1 = in_sub(c, j1m - (j1m / n) * n) ? m23 : 0u;
      const unsigned b0 = load4(c.phase, j1 / n, LL, o00, o01, o10, o11) & pm0;
      const unsigned b1 = load4(c.phase, j1m / n, LL, o00, o01, o10, o11) & pm1;
      double a[3] = {0.0, 0.0, 0.0};
      for (int l = 0; l < c.layers; ++l) {
        const unsigned m = ((b0 >> (8 * l)) & 15u) | (((b1 >> (8 * l)) & 15u) << 4);
#pragma unroll
        for (int d = 0; d < 3; ++d) a[d] += tab[256 * l + m][2 * d];
      }
      const size_t o = (size_t)j1 * NN + (size_t)j2 * N + j3;
      const size_t on[3] = {(size_t)j1p * NN + (size_t)j2 * N + j3, (size_t)j1 * NN + (size_t)j2p * N + j3,
                            (size_t)j1 * NN + (size_t)j2 * N + j3p};
      double g[3][3];  // g[i][d] = D_d psi_i
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double v0 = ps[i][o];
#pragma unroll
        for (int d = 0; d < 3; ++d) g[i][d] = ps[i][on[d]] - v0;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[3 * i + d] = fma(a[d], g[i][d], acc[3 * i + d]);
#pragma unroll
      for (int d = 0; d < 3; ++d) acc[9 + d] += a[d];
      if constexpr (ENERGY) {
        int q = 12;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int jj = i; jj < 3; ++jj) {
            double e = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d)
              e += a[d] * ((i == d ? 1.0 : 0.0) + g[i][d]) * ((jj == d ? 1.0 : 0.0) + g[jj][d]);
            acc[q++] += e;
          }
      }
    }
  }
  double s[18];
  if (reduce_last_block<18>(acc, rb.partials, &rb.st->ticket, s)) {
    if (tid == 0) finalize_scalars(rb.st, FIN_NONE, s, 18);
  }
}

// A_hom sweep: one block per (32 x 8) tile and chunk of planes, about 4 K
// blocks (at most kMaxPartials).
static int ahom_zc(int N) {
  const long long tiles = (long long)((N + 31) / 32) * ((N + 7) / 8);
  int nz = (int)((4096 + tiles - 1) / tiles);
  if (nz > N / 2) nz = N / 2;
  if (nz < 1) nz = 1;
  return (N + nz - 1) / nz;
}

cudaError_t launch_ahom(const CellsDev &c, const double *p0, const double *p1, const double *p2, RedBuf rb,
                        bool energy, cudaStream_t s) {
  const int N = c.N;
  const int zc = ahom_zc(N);
  dim3 grid((N + 31) / 32, (N + 7) / 8, (N + zc - 1) / zc);
  if ((long long)grid.x * grid.y * grid.z > kMaxPartials) return cudaErrorInvalidConfiguration;
  const size_t smem = tab_bytes<double>(c.layers);
  auto kern = energy ? k_ahom<true> : k_ahom<false>;
  const cudaError_t e = allow_dynamic_smem((const void *)kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, dim3(32, 8, 1), smem, s>>>(c, p0, p1, p2, rb, zc);
  return cudaGetLastError();
}

// ------------------------------------------------------------- vector kernels
template <typename T>
__global__ void __launch_bounds__(kThreads) k_x_final_sum(T *__restrict__ x, const T *__restrict__ p, RedBuf rb,
                                                          long long n) {
  const int pend = rb.st->x_pending;
  const T alpha = (T)rb.st->alpha;
  Accum<T> acc;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    T v = x[i];
    if (pend) {
      v = fma(alpha, p[i], v);
      x[i] = v;
    }
    acc.add(v);
  }
  typename Accum<T>::Part vv[1] = {acc.part()};
  double s[1];
  if (reduce_last_block<1>(vv, rb.partials, &rb.st->ticket, s)) {
    if (threadIdx.x == 0) {
      rb.st->red[0] = s[0];
      rb.st->mean = s[0] / (double)n;
      rb.st->x_pending = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_sub_mean(T *__restrict__ x, const Scalars *st, long long n) {
  const T m = (T)st->mean;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    x[i] -= m;
}

static int vec_grid(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  const long long cap = 152 * 16;
  return (int)(g < cap ? g : cap);
}

template <typename T>
cudaError_t launch_x_final_sum(T *x, const T *p, RedBuf rb, long long n, cudaStream_t s) {
  k_x_final_sum<T><<<vec_grid(n), kThreads, 0, s>>>(x, p, rb, n);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_sub_mean(T *x, RedBuf rb, long long n, cudaStream_t s) {
  k_sub_mean<T><<<vec_grid(n), kThreads, 0, s>>>(x, rb.st, n);
  return cudaGetLastError();
}
template cudaError_t launch_x_final_sum<double>(double *, const double *, RedBuf, long long, cudaStream_t);
template cudaError_t launch_x_final_sum<float>(float *, const float *, RedBuf, long long, cudaStream_t);
template cudaError_t launch_sub_mean<double>(double *, RedBuf, long long, cudaStream_t);
template cudaError_t launch_sub_mean<float>(float *, RedBuf, long long, cudaStream_t);

__global__ void __launch_bounds__(kThreads) k_add_f32_to_f64(double *__restrict__ x, const float *__restrict__ d,
                                                             long long n) {
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    x[i] += (double)d[i];
}

cudaError_t launch_add_f32_to_f64(double *x, const float *d, long long n, cudaStream_t s) {
  k_add_f32_to_f64<<<vec_grid(n), kThreads, 0, s>>>(x, d, n);
  return cudaGetLastError();
}

}  // namespace sq
