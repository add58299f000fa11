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
// and the diagonal; no N^3 coefficient field exists.
//
// RHS (Eq. 8 in grid units): b_dir(j) = a_dir(j) - a_dir(j - e_dir).
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

__global__ void k_coeff_gen(uint8_t *__restrict__ phase, int ncell, uint64_t seed, uint64_t thr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncell) phase[i] = ((splitmix64_output(seed, (uint64_t)i) >> 11) < thr) ? 1 : 0;
}

cudaError_t launch_coeff_gen(uint8_t *phase, int L, uint64_t seed, uint64_t thr, cudaStream_t s) {
  int ncell = L * L * L;
  k_coeff_gen<<<(ncell + 255) / 256, 256, 0, s>>>(phase, ncell, seed, thr);
  return cudaGetLastError();
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
template <typename Ti, typename To, int MODE, int RPT>
__global__ void __launch_bounds__(kThreads) k_stencil(CellsDev c, int dir, const Ti *__restrict__ x,
                                                      To *__restrict__ y, RedBuf rb, int fin, int check_done,
                                                      int zc, int nitems) {
  if (check_done && *(volatile int *)&rb.st->done) return;
  __shared__ Ti tab[256][kTabStride];
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
      stencil_rows<Ti, To, MODE, RPT>(c, dir, x, y, tab, cellof, j3, j2b, z0, z1, acc0, acc1);
  }
  typename Accum<Ti>::Part v[2] = {acc0.part(), acc1.part()};
  double s[2];
  if (reduce_last_block<2>(v, rb.partials, &rb.st->ticket, s)) {
    if (tid == 0) finalize_scalars(rb.st, fin, s, 2);
  }
}

// Blocks that fit on the device at once for one kernel (cached per kernel and
// device); 0 on error.
static int resident_blocks(const void *kern, int threads, size_t smem) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  struct Entry {
    const void *k;
    int dev;
    int blocks;
  };
  static Entry cache[64];
  static int used = 0;
  for (int i = 0; i < used; ++i)
    if (cache[i].k == kern && cache[i].dev == dev) return cache[i].blocks;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int blocks = per_sm * sms;
  if (used < 64) cache[used++] = Entry{kern, dev, blocks};
  return blocks;
}

// ------------------------------------------------- staged FP32 operator
// q = A p with p.q for FP32 single solves where N is a multiple of 32 and x is
// 16-byte aligned. A block owns one tile of 32 node columns (j3) x 32 node
// rows (j2) and a run of zc consecutive planes j1 (grid = tiles x plane runs,
// sized to one wave of resident blocks, so the copy pipeline is filled once
// per block). Each plane of the tile with its one-node halo (rows j2-1 and
// j2+32, columns j3-1 and j3+32, periodic) is copied into a ring of kStages
// shared-memory slots with cp.async, kStages - 2 planes ahead of its use: no
// thread waits on HBM latency, and every neighbour is a conflict-free shared-
// memory read at a fixed offset. A thread owns column j3 of four consecutive
// rows; x(j1-1) and x(j1) stay in registers, and so do the four rows'
// coefficients between cell boundaries.
constexpr int kStages = 6;
constexpr int kSW = 40;             // slot row stride (floats): left halo at 3, body 4..35, right halo 36
constexpr int kSRows = 34;          // rows j2-1 .. j2+32
constexpr int kSlot = kSRows * kSW;  // floats per slot

__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// Issues the copies of plane j1 (< N) of tile (j2_0, j3_0) with its halo into slot s.
__device__ __forceinline__ void stage_plane(float *s, const float *__restrict__ x, int N, int j1, int j2_0, int j3_0,
                                            int tid) {
  const float *pl = x + (size_t)j1 * N * N;
  {  // body: 32 rows x 8 chunks of 4 floats, one chunk per thread
    const int row = tid >> 3, ch = tid & 7;
    cp_async16(s + (1 + row) * kSW + 4 + 4 * ch, pl + (size_t)(j2_0 + row) * N + j3_0 + 4 * ch);
  }
  if (tid < 16) {  // halo rows j2_0 - 1 and j2_0 + 32
    const int hr = tid >> 3, ch = tid & 7;
    const int gr = hr ? (j2_0 + 32 == N ? 0 : j2_0 + 32) : (j2_0 == 0 ? N - 1 : j2_0 - 1);
    cp_async16(s + (hr ? kSRows - 1 : 0) * kSW + 4 + 4 * ch, pl + (size_t)gr * N + j3_0 + 4 * ch);
  } else if (tid < 80) {  // halo columns j3_0 - 1 and j3_0 + 32
    const int e = tid - 16, side = e >> 5, row = e & 31;
    const int gc = side ? (j3_0 + 32 == N ? 0 : j3_0 + 32) : (j3_0 == 0 ? N - 1 : j3_0 - 1);
    cp_async4(s + (1 + row) * kSW + (side ? 36 : 3), pl + (size_t)(j2_0 + row) * N + gc);
  }
}

__global__ void __launch_bounds__(kThreads) k_stencil_staged(CellsDev c, const float *__restrict__ x,
                                                             float *__restrict__ y, RedBuf rb, int fin,
                                                             int check_done, int zc, int ntiles) {
  if (check_done && *(volatile int *)&rb.st->done) return;
  extern __shared__ __align__(16) float ring[];  // kStages slots of kSlot floats
  __shared__ float tab[256][kTabStride];
  __shared__ short cellof[kMaxN];
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const int N = c.N, n = c.n, L = c.L, LL = L * L;
  const int NN = N * N;
  const int nbx = N / 32;
  const int tile = blockIdx.x % ntiles, zb = blockIdx.x / ntiles;
  const int j3_0 = (tile % nbx) * 32, j2_0 = (tile / nbx) * 32;
  const int z0 = zb * zc, z1 = min(z0 + zc, N);
  // prologue: planes z0 .. z0 + kStages - 2 (one commit group each, empty past z1)
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    const int j = z0 + st;
    if (j <= z1) stage_plane(ring + st * kSlot, x, N, j == N ? 0 : j, j2_0, j3_0, tid);
    cp_async_commit();
  }
  build_pattern_table<float>(tab, c, tid);
  build_cellof(cellof, N, n, tid);
  __syncthreads();

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j3 = j3_0 + tx, j2b = j2_0 + 4 * ty;
  const int j3m = (j3 == 0) ? N - 1 : j3 - 1;
  const int c3a = cellof[j3], c3b = cellof[j3m];
  int crow[5];
#pragma unroll
  for (int q = 0; q <= 4; ++q) crow[q] = cellof[(j2b - 1 + q < 0) ? N - 1 : j2b - 1 + q] * L;
  const int j1m0 = (z0 == 0) ? N - 1 : z0 - 1;
  int cpos = z0 - cellof[z0] * n;
  unsigned np[4], nc[4];
  row_nibbles<4>(c.phase, cellof[j1m0], LL, crow, c3a, c3b, np);
  if (cpos == 0) {
    row_nibbles<4>(c.phase, cellof[z0], LL, crow, c3a, c3b, nc);
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) nc[r] = np[r];
  }
  float t[4][7];
  row_coeffs<float, 4>(tab, nc, np, t);
  const int row0 = j2b * N + j3;
  float xm[4], x0[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) xm[r] = x[(size_t)j1m0 * NN + row0 + r * N];

  Accum<float> acc;
  for (int k = 0; z0 + k < z1; ++k) {
    const int j1 = z0 + k;
    cp_async_wait<kStages - 3>();  // this thread's copies of planes j1, j1 + 1 have landed
    __syncthreads();               // ... everyone's; and everyone is done with plane j1 - 1's slot
    {
      const int j = j1 + kStages - 1;
      if (j <= z1) stage_plane(ring + ((k + kStages - 1) % kStages) * kSlot, x, N, j == N ? 0 : j, j2_0, j3_0, tid);
      cp_async_commit();
    }
    if (k > 0) {
      cpos = (cpos + 1 == n) ? 0 : cpos + 1;
      if (cpos <= 1) {
#pragma unroll
        for (int r = 0; r < 4; ++r) np[r] = nc[r];
        if (cpos == 0) row_nibbles<4>(c.phase, cellof[j1], LL, crow, c3a, c3b, nc);
        row_coeffs<float, 4>(tab, nc, np, t);
      }
    }
    const float *S0 = ring + (k % kStages) * kSlot + (1 + 4 * ty) * kSW + 4 + tx;
    const float *S1 = ring + ((k + 1) % kStages) * kSlot + (1 + 4 * ty) * kSW + 4 + tx;
    if (k == 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) x0[r] = S0[r * kSW];
    }
    float xp[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) xp[r] = S1[r * kSW];
    float *yp = y + (size_t)j1 * NN + row0;
    float psum = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float *cr = S0 + r * kSW;
      const float x2m = (r == 0) ? cr[-kSW] : x0[r > 0 ? r - 1 : 0];
      const float x2p = (r == 3) ? cr[kSW] : x0[r < 3 ? r + 1 : 3];
      float off = t[r][0] * xp[r];
      off = fmaf(t[r][1], xm[r], off);
      off = fmaf(t[r][2], x2p, off);
      off = fmaf(t[r][3], x2m, off);
      off = fmaf(t[r][4], cr[1], off);
      off = fmaf(t[r][5], cr[-1], off);
      const float ax = fmaf(t[r][6], x0[r], -off);
      yp[r * N] = ax;
      psum = fmaf(x0[r], ax, psum);
    }
    acc.add(psum);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      xm[r] = x0[r];
      x0[r] = xp[r];
    }
  }
  cp_async_wait<0>();
  FF v[2] = {acc.part(), FF{0.f, 0.f}};
  double sres[2];
  if (reduce_last_block<2>(v, rb.partials, &rb.st->ticket, sres)) {
    if (tid == 0) finalize_scalars(rb.st, fin, sres, 2);
  }
}

static cudaError_t launch_stencil_staged(const CellsDev &c, const float *x, float *y, RedBuf rb, int fin,
                                         bool check_done, cudaStream_t s) {
  const int N = c.N;
  const size_t smem = (size_t)kStages * kSlot * sizeof(float);
  const cudaError_t e = cudaFuncSetAttribute(k_stencil_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ntiles = (N / 32) * (N / 32);
  const int resident = resident_blocks((const void *)k_stencil_staged, kThreads, smem);
  if (resident <= 0) return cudaErrorInvalidConfiguration;
  int nz = resident / ntiles;
  if (nz > N / 4) nz = N / 4;  // at least 4 planes per block
  if (nz < 1) nz = 1;
  const int zc = (N + nz - 1) / nz;
  nz = (N + zc - 1) / zc;
  const long long grid = (long long)ntiles * nz;
  if (grid > kMaxPartials) return cudaErrorInvalidConfiguration;
  k_stencil_staged<<<(int)grid, dim3(32, 8, 1), smem, s>>>(c, x, y, rb, fin, check_done ? 1 : 0, zc, ntiles);
  return cudaGetLastError();
}

static int g_planes_override[kMaxN + 1] = {0};
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

template <typename Ti, typename To, int MODE, int RPT>
static cudaError_t launch_stencil_mode(const CellsDev &c, int dir, const Ti *x, To *y, RedBuf rb, int fin,
                                       bool check_done, cudaStream_t s) {
  const int N = c.N;
  const int zc = stencil_zc(N, RPT);
  const long long items =
      (long long)((N + 31) / 32) * ((N + 8 * RPT - 1) / (8 * RPT)) * ((N + zc - 1) / zc);
  auto kern = k_stencil<Ti, To, MODE, RPT>;
  long long grid = resident_blocks((const void *)kern, kThreads, 0);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  if (grid > items) grid = items;
  if (grid > kMaxPartials) grid = kMaxPartials;
  kern<<<(int)grid, dim3(32, 8, 1), 0, s>>>(c, dir, x, y, rb, fin, check_done ? 1 : 0, zc, (int)items);
  return cudaGetLastError();
}

template <typename Ti, typename To, int MODE>
static cudaError_t launch_stencil_rows(const CellsDev &c, int dir, const Ti *x, To *y, RedBuf rb, int fin,
                                       bool check_done, cudaStream_t s) {
  if constexpr (sizeof(Ti) == 4) {
    const int per_n = (c.N >= 8 && c.N <= kMaxN) ? g_rows_override[c.N] : 0;
    const int want = per_n ? per_n : (g_stencil_rows ? g_stencil_rows : 8);
    if constexpr (MODE == ST_MATVEC && sizeof(To) == 4) {
      if (want == 8 && c.N % 32 == 0 && ((uintptr_t)x & 15) == 0)
        return launch_stencil_staged(c, x, y, rb, fin, check_done, s);
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
__global__ void __launch_bounds__(kThreads) k_ahom(CellsDev c, const double *__restrict__ p0,
                                                   const double *__restrict__ p1, const double *__restrict__ p2,
                                                   RedBuf rb, int zc) {
  __shared__ double tab[256][kTabStride];
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
    const double *ps[3] = {p0, p1, p2};
    for (int j1 = z0; j1 < z1; ++j1) {
      const int j1m = (j1 == 0) ? N - 1 : j1 - 1, j1p = (j1 == N - 1) ? 0 : j1 + 1;
      const unsigned m = load4(c.phase, j1 / n, LL, o00, o01, o10, o11) |
                         (load4(c.phase, j1m / n, LL, o00, o01, o10, o11) << 4);
      const double a[3] = {tab[m][0], tab[m][2], tab[m][4]};
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
                        cudaStream_t s) {
  const int N = c.N;
  const int zc = ahom_zc(N);
  dim3 grid((N + 31) / 32, (N + 7) / 8, (N + zc - 1) / zc);
  if ((long long)grid.x * grid.y * grid.z > kMaxPartials) return cudaErrorInvalidConfiguration;
  k_ahom<<<grid, dim3(32, 8, 1), 0, s>>>(c, p0, p1, p2, rb, zc);
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
