// Learned warm start: a periodic 3D convolutional net maps the coefficient
// field to a first guess of the three correctors (an addition to the paper's
// method; the PCG solve keeps judging the guess by its residual).
//
// Net: 6 layers of 3x3x3 periodic convolutions, 32 channels, GELU after the
// first five; input 1 channel (the voxel coefficient, +1 high / -1 low),
// output 3 channels (psi_1..3 / out_scale). Activations are BF16 in
// channel-last layout [sample][voxel][32] (voxel = x3 + N x2 + N^2 x1), weights
// BF16, accumulation FP32.
//
// Kernels:
//  * conv_tc: the 32 -> 32 channel convolutions (forward and data gradient)
//    as direct convolutions on the 5th-generation tensor cores (tcgen05.mma,
//    accumulators in tensor memory; described at the kernel);
//  * conv_mma: implicit GEMM on the tensor cores (mma.sync m16n8k16 BF16, FP32
//    accumulate). Block = 2 x 4 x 32 output voxels, one warp per 32-voxel row
//    (two 16-row m-tiles) and all output channels; the input halo tile
//    (4 x 6 x 34 voxels) and the weights sit in shared memory with padded row
//    strides (conflict-free fragment loads). Epilogues: bias + GELU (stores
//    pre-activation and activation), bias only (FP32 output channels), or
//    plain (data gradient). The data gradient of a layer is the same
//    convolution with the weights flipped in space and transposed in channels.
//  * dw_mma: weight gradients of the 32-channel layers on the tensor cores
//    (mma.sync m16n8k16, operands gathered from channel-last tiles by
//    transposing ldmatrix, one block per (voxel chunk, dz) with its nine taps).
//  * conv_in (layer 1, one input channel), its weight gradient (dw_in) and
//    the bias gradients (db) run on the FP32 pipes; every weight gradient is
//    reduced over the chunks in a fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace sq {
namespace {

constexpr int kC = 32;       // hidden channels
constexpr int kTaps = 27;
constexpr int kLayers = 6;
constexpr int TZ = 2, TY = 4, TX = 32;  // output tile per block (8 warps)
constexpr int HZ = TZ + 2, HY = TY + 2, HX = TX + 2;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ int wrap(int i, int N) { return i < 0 ? i + N : (i >= N ? i - N : i); }

enum Epi { EPI_GELU = 0, EPI_OUT = 1, EPI_PLAIN = 2 };

// out = conv(in, W) over one output tile. CIN in {16, 32} input channels (the
// stored channel count of `in` is CSTR), COUT in {8, 32}. Weights wt are
// [tap][COUT][CIN] BF16 (input channel fastest).
template <int CIN, int CSTR, int COUT, int EPI>
__global__ void __launch_bounds__(256) k_conv_mma(const __nv_bfloat16 *__restrict__ in,
                                                  const __nv_bfloat16 *__restrict__ wt,
                                                  const float *__restrict__ bias, __nv_bfloat16 *__restrict__ zout,
                                                  __nv_bfloat16 *__restrict__ aout, float *__restrict__ fout,
                                                  float out_scale, int N) {
  constexpr int VW = CIN / 2 + 4;   // 32-bit words per staged voxel (padded: conflict-free)
  constexpr int WW = CIN / 2 + 4;   // words per staged weight row
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t *s_in = sm;                          // HZ*HY*HX voxels x VW words
  uint32_t *s_w = sm + HZ * HY * HX * VW;       // 27*COUT rows x WW words
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ntx = N / TX, nty = N / TY, ntz = N / TZ;
  int b = blockIdx.x;
  const int tx = b % ntx; b /= ntx;
  const int ty = b % nty; b /= nty;
  const int tz = b % ntz; b /= ntz;
  const int sample = b;
  const size_t NN = (size_t)N * N, N3 = NN * N;
  const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
  // weights -> smem
  for (int e = tid; e < kTaps * COUT * (CIN / 2); e += 256) {
    const int row = e / (CIN / 2), w = e - row * (CIN / 2);
    s_w[row * WW + w] = reinterpret_cast<const uint32_t *>(wt)[e];
  }
  // input halo tile -> smem (periodic)
  const uint32_t *gin = reinterpret_cast<const uint32_t *>(in) + (size_t)sample * N3 * (CSTR / 2);
  for (int e = tid; e < HZ * HY * HX * (CIN / 2); e += 256) {
    const int v = e / (CIN / 2), w = e - v * (CIN / 2);
    const int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
    const int gx = wrap(x0 + hx - 1, N), gy = wrap(y0 + hy - 1, N), gz = wrap(z0 + hz - 1, N);
    s_in[v * VW + w] = gin[((size_t)gz * NN + (size_t)gy * N + gx) * (CSTR / 2) + w];
  }
  __syncthreads();
  const int g = lane >> 2, t4 = lane & 3;
  const int wz = warp / TY, wy = warp % TY;  // warp's output row: (z0+wz, y0+wy, x0..x0+31)
  constexpr int NT = COUT / 8;
  float acc[2][NT][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[m][nt][i] = 0.f;
  for (int tap = 0; tap < kTaps; ++tap) {
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const int hbase = ((wz + dz) * HY + (wy + dy)) * HX + dx;
#pragma unroll
    for (int kc = 0; kc < CIN / 16; ++kc) {
      uint32_t af[2][4];
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int v0 = hbase + m * 16 + g;
        af[m][0] = s_in[v0 * VW + kc * 8 + t4];
        af[m][1] = s_in[(v0 + 8) * VW + kc * 8 + t4];
        af[m][2] = s_in[v0 * VW + kc * 8 + 4 + t4];
        af[m][3] = s_in[(v0 + 8) * VW + kc * 8 + 4 + t4];
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int row = tap * COUT + nt * 8 + g;
        uint32_t bf[2];
        bf[0] = s_w[row * WW + kc * 8 + t4];
        bf[1] = s_w[row * WW + kc * 8 + 4 + t4];
        mma16816(acc[0][nt], af[0], bf);
        mma16816(acc[1][nt], af[1], bf);
      }
    }
  }
  // epilogue
  const int z = z0 + wz, y = y0 + wy;
#pragma unroll
  for (int m = 0; m < 2; ++m) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int x = x0 + m * 16 + g + half * 8;
      const size_t vox = (size_t)z * NN + (size_t)y * N + x;
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int co = nt * 8 + 2 * t4;
        float v0 = acc[m][nt][half * 2 + 0], v1 = acc[m][nt][half * 2 + 1];
        if (EPI != EPI_PLAIN) {  // bias has COUT entries, or 3 for the output layer
          const int nb = (EPI == EPI_OUT) ? 3 : COUT;
          if (co < nb) v0 += bias[co];
          if (co + 1 < nb) v1 += bias[co + 1];
        }
        if (EPI == EPI_GELU) {
          const size_t o = ((size_t)sample * N3 + vox) * COUT + co;
          *reinterpret_cast<__nv_bfloat162 *>(zout + o) = __floats2bfloat162_rn(v0, v1);
          *reinterpret_cast<__nv_bfloat162 *>(aout + o) = __floats2bfloat162_rn(gelu(v0), gelu(v1));
        } else if (EPI == EPI_PLAIN) {
          const size_t o = ((size_t)sample * N3 + vox) * COUT + co;
          *reinterpret_cast<__nv_bfloat162 *>(aout + o) = __floats2bfloat162_rn(v0, v1);
        } else {  // EPI_OUT: channels 0..2 -> FP32 fields [sample][channel][voxel]
          if (co < 3) fout[((size_t)sample * 3 + co) * N3 + vox] = v0 * out_scale;
          if (co + 1 < 3) fout[((size_t)sample * 3 + co + 1) * N3 + vox] = v1 * out_scale;
        }
      }
    }
  }
}

// ------------------------------------------------- tcgen05 direct convolution
// The 32 -> 32 channel convolutions on the 5th-generation tensor cores, with
// no im2col copy. A CTA tile is 8 (x) x 16 (y) x TZC (z) output voxels of one
// sample. Its input halo, 10 x 18 x (TZC + 2) voxels with periodic wrap, is
// staged once in shared memory as four planes of 8 channels (16 bytes per
// voxel; x fastest, then y, then z). One z-plane of the tile is one M = 128
// operand, row r = x + 8 y. In the no-swizzle K-major layout an 8-row group
// is 8 consecutive 16-byte rows (here 8 consecutive x), and consecutive groups
// (consecutive y) sit one halo row, 160 bytes, apart. So for every tap
// (dz, dy, dx) and 16-channel half kc the A operand is the halo itself, read
// through a descriptor whose start address carries the tap's offset (SBO =
// 160 B between y rows, LBO = the plane stride between the two 8-channel
// halves of K). Per plane, D[128 x 32] = sum over 27 taps and 2 halves of
// A[128 x 16] W[32 x 16]^T: 54 tcgen05.mma (M = 128, N = 32, K = 16) into 32
// TMEM columns. The weights are put in shared memory once per CTA (54 chunks
// of 32 x 16, 1 KB each: SBO 128 B, LBO 512 B).
// The CTA is persistent over its tiles, with two halo buffers and two sets of
// accumulators, and its warps have roles that meet on mbarriers only:
//  * warp 0, one thread: waits until halo b is full and accumulator set b is
//    drained, issues the tile's MMAs (fully unrolled per plane) and commits
//    them to done[b];
//  * warps 1-3 (staging): wait until the MMAs of the tile two back are done
//    (buffer b free), stage the halo by cp.async, wait for their copies,
//    fence them to the tensor core's view and arrive on full[b];
//  * warps 4-11 (read-out): wait on done[b], read accumulator set b (warp w
//    reads TMEM lanes 32 (w % 4) .. of every second plane), add the bias and
//    apply GELU (EPI_GELU: stores z and a) or store the plain sum
//    (EPI_PLAIN), and arrive on drained[b].
// Every wait is bounded and gives up early once another role has given up:
// *err is set, every role stops, the CTA waits for the MMAs it issued and
// frees its TMEM.
constexpr int kTcThreads = 384;
constexpr int kTcStageThreads = 96;  // warps 1-3
constexpr int kTcReadWarps = 8;      // warps 4-11
// weights of a layer with COUT output channels: 54 chunks (tap, K half) of
// COUT rows x 16 input channels
__host__ __device__ constexpr int tc_weight_bytes(int cout) { return 27 * 2 * cout * 32; }
template <int TZC, int COUT = 32>
struct TcTile {
  static constexpr int HV = (TZC + 2) * 18 * 10;                   // halo voxels
  static constexpr int Plane = (HV * 16 + 127) / 128 * 128 + 32;   // bytes, 32 mod 128: conflict-free staging
  static constexpr int Buf = 4 * Plane;                            // one halo: 4 planes of 8 channels
  static constexpr int Smem = 2 * Buf + tc_weight_bytes(COUT) + 1024;  // + 1 KB of alignment slack
  static constexpr int Cols = 2 * TZC * COUT;                           // two accumulator sets
  static_assert(Cols >= 32 && (Cols & (Cols - 1)) == 0, "TMEM allocation: a power of two >= 32 columns");
  // the last byte an A descriptor can reach (plane 2 kc + 1, last z-plane, tap
  // (2, 2, 2), row 127, k 15) stays inside its halo buffer
  static_assert(2 * Plane + ((TZC + 1) * 18 + 2) * 160 + 32 + 15 * 160 + Plane + 7 * 16 + 14 < Buf, "halo extent");
  static_assert(kTcStageThreads >= 80, "staging: 20 threads per piece, 4 pieces");
};

// COUT = 16 with EPI_OUT is the output layer: weights [tap][wrows][32] with
// rows >= wrows zero, bias and out_scale for channels 0..2, FP32 fields
// fout[sample][channel][voxel].
template <int EPI, int TZC, int COUT = 32>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const __nv_bfloat16 *__restrict__ in,
                                                           const __nv_bfloat16 *__restrict__ wt,
                                                           const float *__restrict__ bias,
                                                           __nv_bfloat16 *__restrict__ zout,
                                                           __nv_bfloat16 *__restrict__ aout, int N, int ntiles,
                                                           int wait_polls, int *__restrict__ err,
                                                           float *__restrict__ fout = nullptr, float out_scale = 1.f,
                                                           int wrows = 32) {
  using T = TcTile<TZC, COUT>;
  static_assert(COUT == 32 || (COUT == 16 && EPI == EPI_OUT), "32-channel layers, or the output layer");
  constexpr int kChunk = COUT * 32, kLbo = COUT * 16;  // weight chunk bytes; offset of its second K half
  extern __shared__ __align__(1024) unsigned char smc[];
  __shared__ __align__(8) unsigned long long full[2], done[2], drained[2];
  __shared__ unsigned tmem_base;
  __shared__ volatile int s_fail;
  __shared__ float s_bias[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *wsm = smc + 2 * T::Buf;
  if (EPI == EPI_GELU && tid < 32) s_bias[tid] = bias[tid];
  if (EPI == EPI_OUT && tid < 3) s_bias[tid] = bias[tid];
  // weights [tap][cout][cin] -> chunk (tap, cin half): row n = cout, 16-byte pieces of 8 cin
  for (int e = tid; e < 27 * COUT * 4; e += kTcThreads) {
    const int tap = e / (COUT * 4), r = e - tap * (COUT * 4), n = r >> 2, g8 = r & 3;
    const uint4 v = (n < wrows) ? *reinterpret_cast<const uint4 *>(wt + ((size_t)(tap * wrows + n) * 32 + g8 * 8))
                                : make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(wsm + (tap * 2 + (g8 >> 1)) * kChunk + (n >> 3) * 128 + (g8 & 1) * kLbo +
                               (n & 7) * 16) = v;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, T::Cols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init_count(&full[b], kTcStageThreads);
      tc::mbar_init_count(&done[b], 1);
      tc::mbar_init_count(&drained[b], kTcReadWarps);
    }
    s_fail = 0;
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // weights -> the tensor core's view
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const unsigned tmem = tmem_base;
  const unsigned smc_s = tc::smem_u32(smc);
  const int ntx = N >> 3, nty = N >> 4, ntz = N / TZC;
  const size_t N3 = (size_t)N * N * N;
  const int my_tiles = (ntiles > (int)blockIdx.x) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // origin of this CTA's tile t (tiles run x fastest, then y, z, sample)
  auto origin = [&](int t, int &smp, int &x0, int &y0, int &z0) {
    int b = (int)blockIdx.x + t * (int)gridDim.x;
    x0 = (b % ntx) * 8;
    b /= ntx;
    y0 = (b % nty) * 16;
    b /= nty;
    z0 = (b % ntz) * TZC;
    smp = b / ntz;
  };
  int last = -1;  // (warp 0, lane 0) the last tile whose MMAs were issued
  if (warp == 0) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
      // descriptors: the start address (>> 4) sits in the low 14 bits and no
      // offset carries out of them (shared addresses < 256 KB), so a tap's
      // offset is added to the low word only
      const uint64_t b64 = tc::sdesc(tc::smem_u32(wsm), (unsigned)kLbo, 128u);
      const uint32_t b_lo = (uint32_t)b64, b_hi = (uint32_t)(b64 >> 32);
      for (int t = 0; t < my_tiles; ++t) {
        const int b = t & 1;
        if (!tc::mbar_wait_or_fail(&full[b], (unsigned)(t >> 1) & 1u, wait_polls, &s_fail)) {
          s_fail = 1;
          break;
        }
        if (t >= 2 && !tc::mbar_wait_or_fail(&drained[b], (unsigned)((t - 2) >> 1) & 1u, wait_polls, &s_fail)) {
          s_fail = 1;
          break;
        }
        tc::fence_after_sync();
        const uint64_t a64 = tc::sdesc(smc_s + (unsigned)b * T::Buf, T::Plane, 160u);
        const uint32_t a_hi = (uint32_t)(a64 >> 32);
        const unsigned d0 = tmem + (unsigned)b * (TZC * COUT);
#pragma unroll 1
        for (int zl = 0; zl < TZC; ++zl) {
          const uint32_t a_lo = (uint32_t)a64 + (uint32_t)(zl * (18 * 160 / 16));
#pragma unroll
          for (int tap = 0; tap < 27; ++tap) {
#pragma unroll
            for (int kc = 0; kc < 2; ++kc) {
              const uint32_t aoff = (uint32_t)((((tap / 9) * 18 + (tap / 3) % 3) * 160 + (tap % 3) * 16 +
                                                kc * 2 * T::Plane) >> 4);
              const uint32_t boff = (uint32_t)((tap * 2 + kc) * (kChunk >> 4));
              tc::mma_bf16(d0 + zl * COUT, ((uint64_t)a_hi << 32) | (a_lo + aoff),
                           ((uint64_t)b_hi << 32) | (b_lo + boff), idesc, (tap | kc) ? 1u : 0u);
            }
          }
        }
        tc::mma_commit(&done[b]);
        last = t;
      }
    }
  } else if (warp < 4) {
    // staging: thread st copies piece g8 = st % 4 (channels 8 g8 ..) of halo
    // column hx = j % 10 (j = st / 4 < 20) in every second halo row (y, z),
    // starting at row j / 10
    const int st = tid - 32, g8 = st & 3, j = st >> 2, hx = j % 10;
    for (int t = 0; t < my_tiles; ++t) {
      const int b = t & 1;
      if (t >= 2 && !tc::mbar_wait_or_fail(&done[b], (unsigned)((t - 2) >> 1) & 1u, wait_polls, &s_fail)) {
        s_fail = 1;
        break;
      }
      if (j < 20) {
        int smp, x0, y0, z0;
        origin(t, smp, x0, y0, z0);
        const __nv_bfloat16 *gs = in + (size_t)smp * N3 * 32 + (size_t)wrap(x0 + hx - 1, N) * 32 + g8 * 8;
        const unsigned dst = smc_s + (unsigned)b * T::Buf + (unsigned)(g8 * T::Plane + hx * 16);
        int hy = j / 10, hz = 0;
#pragma unroll 2
        for (int rr = j / 10; rr < (TZC + 2) * 18; rr += 2) {  // halo row rr = hy + 18 hz
          const int row = wrap(z0 + hz - 1, N) * N + wrap(y0 + hy - 1, N);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + (unsigned)rr * 160u),
                       "l"(gs + (size_t)row * N * 32)
                       : "memory");
          hy += 2;
          if (hy >= 18) {
            hy -= 18;
            ++hz;
          }
        }
      }
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the copies -> the tensor core's view
      tc::mbar_arrive(&full[b]);
    }
  } else {
    // read-out: TMEM lane quarter q, planes h, h + 2, ...
    const int q = warp & 3, h = (warp - 4) >> 2, r = 32 * q + lane;
    for (int t = 0; t < my_tiles; ++t) {
      const int b = t & 1;
      // the warp gives up as one (its TMEM loads are warp-collective)
      const bool ok = tc::mbar_wait_or_fail(&done[b], (unsigned)(t >> 1) & 1u, wait_polls, &s_fail);
      if (!__all_sync(0xffffffffu, ok)) {
        s_fail = 1;
        break;
      }
      tc::fence_after_sync();
      int smp, x0, y0, z0;
      origin(t, smp, x0, y0, z0);
      const size_t row = (size_t)smp * N3 + (size_t)(y0 + (r >> 3)) * N + x0 + (r & 7);
      const unsigned taddr = tmem + ((unsigned)(32 * q) << 16) + (unsigned)b * (TZC * COUT);
#pragma unroll 1
      for (int zl = h; zl < TZC; zl += 2) {
        if constexpr (EPI == EPI_OUT) {
          float v[16];
          tc::tmem_ld_32x16(taddr + zl * COUT, v);
          const size_t vox = row - (size_t)smp * N3 + (size_t)(z0 + zl) * N * N;
#pragma unroll
          for (int co = 0; co < 3; ++co) fout[((size_t)smp * 3 + co) * N3 + vox] = (v[co] + s_bias[co]) * out_scale;
        } else {
        float v[32];
        tc::tmem_ld_32x32(taddr + zl * 32, v);
        const size_t o = (row + (size_t)(z0 + zl) * N * N) * 32;
        uint32_t zw[16], aw[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float z0f = v[2 * k] + (EPI == EPI_GELU ? s_bias[2 * k] : 0.f);
          const float z1f = v[2 * k + 1] + (EPI == EPI_GELU ? s_bias[2 * k + 1] : 0.f);
          __nv_bfloat162 zb = __floats2bfloat162_rn(z0f, z1f);
          zw[k] = *reinterpret_cast<uint32_t *>(&zb);
          if (EPI == EPI_GELU) {
            __nv_bfloat162 ab = __floats2bfloat162_rn(gelu(z0f), gelu(z1f));
            aw[k] = *reinterpret_cast<uint32_t *>(&ab);
          }
        }
        uint4 *zdst = reinterpret_cast<uint4 *>((EPI == EPI_GELU ? zout : aout) + o);
#pragma unroll
        for (int k = 0; k < 4; ++k) zdst[k] = make_uint4(zw[4 * k], zw[4 * k + 1], zw[4 * k + 2], zw[4 * k + 3]);
        if (EPI == EPI_GELU) {
          uint4 *adst = reinterpret_cast<uint4 *>(aout + o);
#pragma unroll
          for (int k = 0; k < 4; ++k) adst[k] = make_uint4(aw[4 * k], aw[4 * k + 1], aw[4 * k + 2], aw[4 * k + 3]);
        }
        }
      }
      tc::fence_before_sync();  // the TMEM reads precede the MMAs that overwrite set b
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&drained[b]);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy into this CTA's memory left in flight
  __syncthreads();
  // the last commit covers every MMA this CTA issued: none may be in flight at exit
  if (tid == 0 && last >= 0 && !tc::mbar_wait(&done[last & 1], (unsigned)(last >> 1) & 1u, 1 << 24)) s_fail = 1;
  tc::fence_before_sync();
  __syncthreads();
  if (s_fail && tid == 0) atomicExch(err, 1);
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, T::Cols);
  }
}

// Layer 1 (one input channel, FP32 feature): z = sum_tap w[tap][co] f + b.
__global__ void __launch_bounds__(256) k_conv_in(const float *__restrict__ f, const float *__restrict__ w,
                                                 const float *__restrict__ bias, __nv_bfloat16 *__restrict__ zout,
                                                 __nv_bfloat16 *__restrict__ aout, int N, long long total) {
  __shared__ __align__(16) float sw[kTaps * kC];  // [tap][co]
  __shared__ float sb[kC];
  for (int e = threadIdx.x; e < kTaps * kC; e += 256) sw[e] = w[e];
  if (threadIdx.x < kC) sb[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  if (i >= total) return;
  const size_t N3 = (size_t)N * N * N;
  const long long sample = i / N3;
  const size_t vox = i - sample * N3;
  const int x = vox % N, y = (vox / N) % N, z = vox / ((size_t)N * N);
  float nb[kTaps];
#pragma unroll
  for (int tap = 0; tap < kTaps; ++tap) {
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    nb[tap] = f[sample * N3 + (size_t)wrap(z + dz, N) * N * N + (size_t)wrap(y + dy, N) * N + wrap(x + dx, N)];
  }
  // eight output channels per round: 16-byte weight reads (a broadcast) and
  // 16-byte stores; each output sums bias + w nb over the taps in tap order
  const float4 *sw4 = reinterpret_cast<const float4 *>(sw);
#pragma unroll 1
  for (int cb = 0; cb < kC / 8; ++cb) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = sb[cb * 8 + k];
#pragma unroll
    for (int tap = 0; tap < kTaps; ++tap) {
      const float4 wa = sw4[tap * (kC / 4) + cb * 2], wb = sw4[tap * (kC / 4) + cb * 2 + 1];
      const float t = nb[tap];
      v[0] = fmaf(wa.x, t, v[0]);
      v[1] = fmaf(wa.y, t, v[1]);
      v[2] = fmaf(wa.z, t, v[2]);
      v[3] = fmaf(wa.w, t, v[3]);
      v[4] = fmaf(wb.x, t, v[4]);
      v[5] = fmaf(wb.y, t, v[5]);
      v[6] = fmaf(wb.z, t, v[6]);
      v[7] = fmaf(wb.w, t, v[7]);
    }
    uint32_t zw[4], aw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      __nv_bfloat162 zb = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
      __nv_bfloat162 ab = __floats2bfloat162_rn(gelu(v[2 * k]), gelu(v[2 * k + 1]));
      zw[k] = *reinterpret_cast<uint32_t *>(&zb);
      aw[k] = *reinterpret_cast<uint32_t *>(&ab);
    }
    const size_t o = (size_t)i * kC + cb * 8;
    *reinterpret_cast<uint4 *>(zout + o) = make_uint4(zw[0], zw[1], zw[2], zw[3]);
    *reinterpret_cast<uint4 *>(aout + o) = make_uint4(aw[0], aw[1], aw[2], aw[3]);
  }
}

// Input feature: voxel coefficient as +1 (high) / -1 (low), from the cell phases.
// +1 where the voxel is high (its cell is high and, with sub-cell inclusions,
// it lies in the cell's inclusion cube [sub_lo, sub_hi)^3), else -1.
__global__ void k_feature(const uint8_t *__restrict__ phase, int L, int n, int sub_lo, int sub_hi,
                          float *__restrict__ f) {
  const int N = L * n;
  const size_t N3 = (size_t)N * N * N;
  const size_t i = blockIdx.x * 256ULL + threadIdx.x;
  if (i >= N3) return;
  const int x = i % N, y = (i / N) % N, z = i / ((size_t)N * N);
  const int ux = x % n, uy = y % n, uz = z % n;
  const bool inside = ux >= sub_lo && ux < sub_hi && uy >= sub_lo && uy < sub_hi && uz >= sub_lo && uz < sub_hi;
  f[i] = (inside && phase[((size_t)(z / n) * L + y / n) * L + x / n]) ? 1.f : -1.f;
}

// FP32 fields [3][N3] -> three FP64 correctors
__global__ void k_to_psi(const float *__restrict__ o, double *p0, double *p1, double *p2, long long N3) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  if (i >= N3) return;
  p0[i] = o[i];
  p1[i] = o[N3 + i];
  p2[i] = o[2 * N3 + i];
}

// ----------------------------------------------------------------- training
// Loss L = sum((y - t)^2) / out_scale^2 over samples x 3 channels x voxels
// (Adam is invariant to the overall gradient scale). Writes dL/d(conv6 out)
// = 2 (y - t) / out_scale as BF16 [sample][voxel][16] (channels 3..15 zero)
// and per-block loss partials.
__global__ void __launch_bounds__(256) k_loss_grad(const float *__restrict__ y, const float *__restrict__ tgt,
                                                   __nv_bfloat16 *__restrict__ g, float inv_scale,
                                                   double *__restrict__ partials, long long N3, int B) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;  // sample * N3 + voxel
  Accum<float> acc;
  if (i < (long long)B * N3) {
    const long long smp = i / N3, vox = i - smp * N3;
    uint32_t w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = 0u;
    for (int c = 0; c < 3; ++c) {
      const float e = (y[(smp * 3 + c) * N3 + vox] - tgt[(smp * 3 + c) * N3 + vox]) * inv_scale;
      acc.add(e * e);
      const __nv_bfloat16 gb = __float2bfloat16_rn(2.f * e);
      const uint32_t bits = (uint32_t)(*reinterpret_cast<const unsigned short *>(&gb));
      w[c >> 1] |= bits << (16 * (c & 1));
    }
    uint4 *dst = reinterpret_cast<uint4 *>(g + i * 16);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
  __shared__ double sh[8];
  double v = warp_sum(acc.get());
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += sh[k];
    partials[blockIdx.x] = t;
  }
}

// e = (y - t) / out_scale, FP32 fields [sample][3][N3]
__global__ void k_err(const float *__restrict__ y, const float *__restrict__ tgt, float *__restrict__ e, float inv_scale,
                      long long n) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  if (i < n) e[i] = (y[i] - tgt[i]) * inv_scale;
}

// r = (a - b) * s, FP32 fields
__global__ void k_sub_scale(const float *__restrict__ a, float *__restrict__ b, float s, long long n) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  if (i < n) b[i] = (a[i] - b[i]) * s;
}

// per-block partial sums of a . b (fixed order inside the block)
__global__ void __launch_bounds__(256) k_dot_partial(const float *__restrict__ a, const float *__restrict__ b,
                                                     double *__restrict__ partials, long long n) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  Accum<float> acc;
  if (i < n) acc.add_prod(a[i], b[i]);
  __shared__ double sh[8];
  double v = warp_sum(acc.get());
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += sh[k];
    partials[blockIdx.x] = t;
  }
}

// dL/d(conv6 out) = 2 A e as channel-last BF16 [sample][voxel][16], channels 0..2
__global__ void k_pack_grad(const float *__restrict__ ae, __nv_bfloat16 *__restrict__ g, long long N3, int B) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;  // sample * N3 + voxel
  if (i >= (long long)B * N3) return;
  const long long smp = i / N3, vox = i - smp * N3;
  uint32_t w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = 0u;
  for (int c = 0; c < 3; ++c) {
    const __nv_bfloat16 gb = __float2bfloat16_rn(2.f * ae[(smp * 3 + c) * N3 + vox]);
    const uint32_t bits = (uint32_t)(*reinterpret_cast<const unsigned short *>(&gb));
    w[c >> 1] |= bits << (16 * (c & 1));
  }
  uint4 *dst = reinterpret_cast<uint4 *>(g + i * 16);
  dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
  dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// gz = ga * gelu'(z), 32 channels BF16; one thread per 8 values (16-byte
// accesses), n8 = values / 8.
__global__ void k_gelu_bwd(const __nv_bfloat16 *__restrict__ ga, const __nv_bfloat16 *__restrict__ z,
                           __nv_bfloat16 *__restrict__ gz, long long n8) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  if (i >= n8) return;
  const uint4 a4 = reinterpret_cast<const uint4 *>(ga)[i];
  const uint4 z4 = reinterpret_cast<const uint4 *>(z)[i];
  const __nv_bfloat162 *a2 = reinterpret_cast<const __nv_bfloat162 *>(&a4);
  const __nv_bfloat162 *z2 = reinterpret_cast<const __nv_bfloat162 *>(&z4);
  uint4 o4;
  __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&o4);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 a = __bfloat1622float2(a2[k]);
    const float2 zz = __bfloat1622float2(z2[k]);
    o2[k] = __floats2bfloat162_rn(a.x * gelu_grad(zz.x), a.y * gelu_grad(zz.y));
  }
  reinterpret_cast<uint4 *>(gz)[i] = o4;
}

// Weight and bias gradient partials of layer 1 (one input channel, the FP32
// feature f): dW[tap][co] = sum_v f[v + off_tap] G[v][co] and dB[co] =
// sum_v G[v][co] over the voxels of one chunk (FP32 pipes). Per tile of 128
// voxels the block stages G transposed (channel rows, padded: conflict-free
// 16-byte reads) and f at the 27 tap offsets of every voxel (slot 27 holds
// ones: the bias); thread (co = lane, slots warp + 8 k) then runs a
// 4 x 4 register block over the voxels. Partials go to the layout
// (chunk, tap, co) that k_dw_reduce sums in a fixed order. The chunk is a
// multiple of 128 voxels (of 4 N, N a multiple of 32).
__global__ void __launch_bounds__(256) k_dw_in(const float *__restrict__ f, const __nv_bfloat16 *__restrict__ G,
                                               int N, long long total, int chunk, float *__restrict__ partials) {
  constexpr int V = 128;
  __shared__ __align__(16) float sf[28][V];
  __shared__ __align__(16) float sg[32][V + 4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long v0 = (long long)blockIdx.x * chunk;
  const long long v1 = (v0 + chunk < total) ? v0 + chunk : total;
  const size_t N3 = (size_t)N * N * N;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (long long vb = v0; vb < v1; vb += V) {
    __syncthreads();  // the previous tile is consumed
    for (int e = tid; e < V * 16; e += 256) {  // G: 128 voxels x 16 channel pairs
      const int vi = e >> 4, c2 = e & 15;
      const float2 g = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(G)[(vb + vi) * 16 + c2]);
      sg[2 * c2][vi] = g.x;
      sg[2 * c2 + 1][vi] = g.y;
    }
    {  // f at the tap offsets: thread = (voxel tid % 128, taps tid / 128 + 2 k)
      const int vi = tid & (V - 1);
      const long long v = vb + vi;
      const long long smp = v / (long long)N3;
      const int vox = (int)(v - smp * (long long)N3);
      const int x = vox % N, y = (vox / N) % N, z = vox / (N * N);
      const float *fs = f + smp * (long long)N3;
      for (int tap = tid >> 7; tap < 28; tap += 2) {
        float val = 1.f;
        if (tap < 27) {
          const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
          val = fs[((size_t)wrap(z + dz, N) * N + wrap(y + dy, N)) * N + wrap(x + dx, N)];
        }
        sf[tap][vi] = val;
      }
    }
    __syncthreads();
#pragma unroll 2
    for (int vi = 0; vi < V; vi += 4) {
      const float4 g = *reinterpret_cast<const float4 *>(&sg[lane][vi]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int tap = warp + 8 * k;
        if (tap < 28) {
          const float4 a = *reinterpret_cast<const float4 *>(&sf[tap][vi]);
          acc[k] = fmaf(a.x, g.x, fmaf(a.y, g.y, fmaf(a.z, g.z, fmaf(a.w, g.w, acc[k]))));
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int tap = warp + 8 * k;
    if (tap < 28) partials[((size_t)blockIdx.x * 28 + tap) * 32 + lane] = acc[k];
  }
}

// Bias gradient partials of a layer with CG output channels stored with
// stride CGS (BF16, a multiple of 8): dB[co] = sum_v G[v][co] over one
// chunk, written to the bias slot (tap 27, input channel 0) of the chunk's
// partials (nout = CG CA entries per tap). Thread t reads the 8 channels
// 8 (t % 4) .. of voxels t / 4 + 64 k (16-byte loads); the 64 voxel lanes are
// added in a fixed order.
__global__ void __launch_bounds__(256) k_db(const __nv_bfloat16 *__restrict__ G, int CGS, int CG, long long total,
                                            int chunk, int nout, int ca, float *__restrict__ partials) {
  __shared__ float red[64][33];
  const int c8 = threadIdx.x & 3, vl = threadIdx.x >> 2;
  const long long v0 = (long long)blockIdx.x * chunk;
  const long long v1 = (v0 + chunk < total) ? v0 + chunk : total;
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.f;
  if (c8 * 8 < CGS) {
#pragma unroll 4
    for (long long v = v0 + vl; v < v1; v += 64) {
      const uint4 g4 = *reinterpret_cast<const uint4 *>(G + v * CGS + c8 * 8);
      const __nv_bfloat162 *g2 = reinterpret_cast<const __nv_bfloat162 *>(&g4);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 g = __bfloat1622float2(g2[k]);
        acc[2 * k] += g.x;
        acc[2 * k + 1] += g.y;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) red[vl][c8 * 8 + k] = acc[k];
  __syncthreads();
  const int co = threadIdx.x;
  if (co < CG) {
    float t = 0.f;
    for (int w = 0; w < 64; ++w) t += red[w][co];
    partials[((size_t)blockIdx.x * 28 + 27) * nout + (size_t)co * ca] = t;
  }
}

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
// Four (two) 8 x 8 b16 matrices from shared memory, transposed: row addresses
// from lanes 0-31 (0-15), 16-byte aligned.
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}

// Weight gradient on the tensor cores (layers with 32 input channels):
// dW[tap][co][ci] = sum_v G[v][co] A[v + off_tap][ci], one GEMM per tap with
// M = co, N = ci and K running over the voxels of the chunk (mma.sync m16n8k16
// BF16, FP32 accumulate). blockIdx.y fixes dz; the block's nine taps (dy, dx)
// share each staged tile. A tile is TY = 4 consecutive x-rows of one plane of
// G (CGM of its CGS channels) and the TY + 2 rows of A around it (plane
// z + dz, periodic), in shared memory with rows padded to 80 (48) bytes so the
// transposing ldmatrix reads are conflict-free. Both operands arrive
// channel-last, so the K pairs of a fragment (two voxels) are gathered by
// ldmatrix .trans; a shifted tap is only a different row address per lane
// (the x wrap included). Warp w owns the fragments f = w + 8 j of the block's
// 9 x NP (m-tile, n-tile) pairs. Partials go to the layout of k_dw
// (chunk, tap, co, ci) for the same fixed-order reduction.
template <int CGM>
__global__ void __launch_bounds__(256) k_dw_mma(const __nv_bfloat16 *__restrict__ A,
                                                const __nv_bfloat16 *__restrict__ G, int CGS, int CG, int N,
                                                long long total, int chunk, float *__restrict__ partials) {
  constexpr int TY = 4;
  constexpr int SA = 40;        // bf16 per staged A row (32 + 8)
  constexpr int SG = CGM + 8;   // bf16 per staged G row
  constexpr int NP = (CGM / 16) * 4;
  constexpr int F = 9 * NP;
  constexpr int J = (F + 7) / 8;
  extern __shared__ __align__(16) __nv_bfloat16 smw[];
  const int TN = TY * N;
  __nv_bfloat16 *sg = smw;                    // [TN][SG]
  __nv_bfloat16 *sa = smw + (size_t)TN * SG;  // [(TY + 2) N][SA]
  const int dz = (int)blockIdx.y - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp % NP, mt = pair / 4, nt = pair % 4;
  const size_t N3 = (size_t)N * N * N;
  float acc[J][4];
#pragma unroll
  for (int j = 0; j < J; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
  const long long v0 = (long long)blockIdx.x * chunk;
  const long long v1 = (v0 + chunk < total) ? v0 + chunk : total;
  for (long long vt = v0; vt < v1; vt += TN) {
    const long long smp = vt / (long long)N3;
    const size_t vox0 = (size_t)(vt - smp * (long long)N3);
    const int z = (int)(vox0 / ((size_t)N * N)), y0 = (int)((vox0 / N) % N);
    __syncthreads();  // the previous tile's fragments are read
    for (int e = threadIdx.x; e < TN * (CGM / 8); e += 256) {
      const int v = e / (CGM / 8), c8 = e - v * (CGM / 8);
      *reinterpret_cast<uint4 *>(sg + (size_t)v * SG + c8 * 8) =
          *reinterpret_cast<const uint4 *>(G + (size_t)(vt + v) * CGS + c8 * 8);
    }
    const int za = wrap(z + dz, N);
    for (int e = threadIdx.x; e < (TY + 2) * N * 4; e += 256) {
      const int v = e >> 2, c8 = e & 3;
      const int rr = v / N, x = v - rr * N;
      const int ya = wrap(y0 - 1 + rr, N);
      *reinterpret_cast<uint4 *>(sa + (size_t)v * SA + c8 * 8) = *reinterpret_cast<const uint4 *>(
          A + ((size_t)smp * N3 + ((size_t)za * N + ya) * N + x) * 32 + c8 * 8);
    }
    __syncthreads();
    for (int kv0 = 0; kv0 < TN; kv0 += 16) {  // 16 voxels of one row (16 | N)
      const int ry = kv0 / N, x0 = kv0 - ry * N;
      uint32_t af[4];
      {
        const int q = lane >> 3, r = lane & 7;
        ldsm_x4_t(af, smem_addr(sg + (size_t)(kv0 + r + 8 * (q >> 1)) * SG + mt * 16 + 8 * (q & 1)));
      }
      const int kk = lane & 15;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int f = warp + 8 * j;
        if (f < F) {
          const int t9 = f / NP, dy = t9 / 3 - 1, dx = t9 % 3 - 1;
          const int xs = wrap(x0 + kk + dx, N);
          uint32_t bf[2];
          ldsm_x2_t(bf, smem_addr(sa + (size_t)((ry + 1 + dy) * N + xs) * SA + nt * 8));
          mma16816(acc[j], af, bf);
        }
      }
    }
  }
  const int g = lane >> 2, t4 = lane & 3;
  const int nout = CG * 32;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int f = warp + 8 * j;
    if (f >= F) continue;
    const int tap = (dz + 1) * 9 + f / NP;
    float *pp = partials + ((size_t)blockIdx.x * 28 + tap) * nout;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int co = mt * 16 + g + 8 * h, ci = nt * 8 + 2 * t4;
      if (co < CG) {
        pp[co * 32 + ci] = acc[j][2 * h];
        pp[co * 32 + ci + 1] = acc[j][2 * h + 1];
      }
    }
  }
}

// Sum of the chunk partials (fixed order) -> weight gradient [27][CG][CA]
// (taps 0..26) and bias gradient [CG] (tap 27, input slot 0).
__global__ void k_dw_reduce(const float *__restrict__ partials, int nchunk, int nout, int ca, float *__restrict__ gw,
                            float *__restrict__ gb) {
  const int o = blockIdx.x * 256 + threadIdx.x;  // over 28 * nout
  if (o >= 28 * nout) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += partials[(size_t)c * 28 * nout + o];
  const int tap = o / nout, r = o - tap * nout;
  if (tap < 27) {
    gw[o] = (float)s;
  } else if (r % ca == 0) {
    gb[r / ca] = (float)s;
  }
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of a layer's FP32 weights [27][cout][cin]: forward layout
// [tap][COUTP][CINP] and data-gradient layout [tap'][CINP2=cin][COUTP2] with
// tap' = 26 - tap (spatial flip) and channels transposed; padding rows zero.
__global__ void k_pack_weights(const float *__restrict__ w, int cout, int cin, int coutp, __nv_bfloat16 *__restrict__ wf,
                               __nv_bfloat16 *__restrict__ wb, int coutp2) {
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int nf = 27 * coutp * cin;
  if (i < nf) {
    const int tap = i / (coutp * cin), r = i - tap * coutp * cin, co = r / cin, ci = r - co * cin;
    wf[i] = __float2bfloat16_rn(co < cout ? w[(tap * cout + co) * cin + ci] : 0.f);
  }
  if (wb) {
    const int nb = 27 * cin * coutp2;
    if (i < nb) {
      const int tp = i / (cin * coutp2), r = i - tp * cin * coutp2, ci = r / coutp2, co = r - ci * coutp2;
      const int tap = 26 - tp;
      wb[i] = __float2bfloat16_rn(co < cout ? w[(tap * cout + co) * cin + ci] : 0.f);
    }
  }
}

__global__ void k_target_f32(const double *__restrict__ t0, const double *__restrict__ t1, const double *__restrict__ t2,
                             float *__restrict__ out, long long N3) {
  const long long i = blockIdx.x * 256LL + threadIdx.x;
  if (i >= N3) return;
  out[i] = (float)t0[i];
  out[N3 + i] = (float)t1[i];
  out[2 * N3 + i] = (float)t2[i];
}

}  // namespace
}  // namespace sq

using namespace sq;

// Parameter layout (FP32 master): per layer l, weights [27][cout][cin] then bias [cout].
struct sq_net {
  int N = 0, max_batch = 0;
  double out_scale = 1.0;
  int cin[kLayers], cout[kLayers];
  long long woff[kLayers], boff[kLayers], nparam = 0;
  float *d_w = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
  __nv_bfloat16 *d_wf[kLayers] = {nullptr}, *d_wb[kLayers] = {nullptr};
  float *d_f = nullptr, *d_y = nullptr, *d_t = nullptr;
  __nv_bfloat16 *d_z[5] = {nullptr}, *d_a[5] = {nullptr};
  __nv_bfloat16 *d_g6 = nullptr, *d_ga = nullptr, *d_gz = nullptr;
  float *d_dwpart = nullptr;
  float *d_e = nullptr, *d_ae = nullptr;  // error field and A e (energy loss)
  Scalars *d_st = nullptr;
  double *d_partials = nullptr;           // reductions of the operator kernel
  double *d_lpart = nullptr, *h_lpart = nullptr;
  int *d_err = nullptr, *h_err = nullptr;  // a bounded wait of the tcgen05 convolution gave up
  int nchunk = 0, chunk = 0;
  int step = 0;
  std::vector<void *> allocs;
};

namespace {

#define SQN_CK(call)                        \
  do {                                      \
    if ((call) != cudaSuccess) return SQ_ECUDA; \
  } while (0)

template <int CIN, int CSTR, int COUT, int EPI>
int conv(const sq_net *net, int B, const __nv_bfloat16 *in, const __nv_bfloat16 *wt, const float *bias,
         __nv_bfloat16 *z, __nv_bfloat16 *a, float *fo, cudaStream_t s) {
  const int N = net->N;
  const size_t smem = (size_t)(HZ * HY * HX * (CIN / 2 + 4) + kTaps * COUT * (CIN / 2 + 4)) * 4;
  auto kern = k_conv_mma<CIN, CSTR, COUT, EPI>;
  SQN_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int blocks = (N / TX) * (N / TY) * (N / TZ) * B;
  kern<<<blocks, 256, smem, s>>>(in, wt, bias, z, a, fo, (float)net->out_scale, N);
  SQN_CK(cudaGetLastError());
  return SQ_OK;
}

// The 32 -> 32 channel convolutions on tcgen05 (SQ_OPT_CONV_TC = 1: tile
// depth chosen below; 2 or 4: that depth) or on mma.sync (0): same inputs,
// outputs and layouts.
int g_conv_tc = 1;

template <int EPI, int TZC, int COUT = 32>
int conv_tc(const sq_net *net, int B, const __nv_bfloat16 *in, const __nv_bfloat16 *wt, const float *bias,
            __nv_bfloat16 *z, __nv_bfloat16 *a, int grid, cudaStream_t s, float *fo = nullptr, int wrows = 32) {
  const int N = net->N;
  const long long ntiles = (long long)B * N * N * N / (128 * TZC);
  auto kern = k_conv_tc<EPI, TZC, COUT>;
  constexpr int smem = TcTile<TZC, COUT>::Smem;
  SQN_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int g = (int)(ntiles < grid ? ntiles : grid);
  kern<<<g, kTcThreads, smem, s>>>(in, wt, bias, z, a, N, (int)ntiles, stage_wait_polls(), net->d_err, fo,
                                    (float)net->out_scale, wrows);
  SQN_CK(cudaGetLastError());
  return SQ_OK;
}

template <int EPI>
int conv32(const sq_net *net, int B, const __nv_bfloat16 *in, const __nv_bfloat16 *wt, const float *bias,
           __nv_bfloat16 *z, __nv_bfloat16 *a, cudaStream_t s) {
  if (!g_conv_tc) return conv<32, 32, 32, EPI>(net, B, in, wt, bias, z, a, nullptr, s);
  // one CTA per SM (the shared memory of either depth allows no second)
  int dev = 0, sms = 0;
  SQN_CK(cudaGetDevice(&dev));
  SQN_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int tz = g_conv_tc;
  if (tz == 1) {
    // depth 4 stages less halo per voxel (6/4 z-planes against 4/2); depth 2
    // balances better when there are few tiles per SM: compare the planes the
    // busiest SM computes, depth 2 charged 10 % for its larger halo
    const long long vox = (long long)B * net->N * net->N * net->N;
    const long long t4 = vox / 512, t2 = vox / 256;
    const double w4 = 4.0 * (double)((t4 + sms - 1) / sms), w2 = 2.2 * (double)((t2 + sms - 1) / sms);
    tz = (w2 < w4) ? 2 : 4;
  }
  return tz == 2 ? conv_tc<EPI, 2>(net, B, in, wt, bias, z, a, sms, s)
                 : conv_tc<EPI, 4>(net, B, in, wt, bias, z, a, sms, s);
}

// The output layer (32 -> 3 channels, FP32 fields times out_scale): on
// tcgen05 with 16 accumulator columns per plane (channels 3..15 zero) where
// the convolutions run there, else on mma.sync. Its packed weights have 8
// rows per tap.
int conv_out(const sq_net *net, int B, const __nv_bfloat16 *in, const __nv_bfloat16 *wt, const float *bias,
             float *fo, cudaStream_t s) {
  if (!g_conv_tc) return conv<32, 32, 8, EPI_OUT>(net, B, in, wt, bias, nullptr, nullptr, fo, s);
  int dev = 0, sms = 0;
  SQN_CK(cudaGetDevice(&dev));
  SQN_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long vox = (long long)B * net->N * net->N * net->N;
  const long long t4 = vox / 512, t2 = vox / 256;
  const double w4 = 4.0 * (double)((t4 + sms - 1) / sms), w2 = 2.2 * (double)((t2 + sms - 1) / sms);
  const int tz = (g_conv_tc == 2 || g_conv_tc == 4) ? g_conv_tc : ((w2 < w4) ? 2 : 4);
  return tz == 2 ? conv_tc<EPI_OUT, 2, 16>(net, B, in, wt, bias, nullptr, nullptr, sms, s, fo, 8)
                 : conv_tc<EPI_OUT, 4, 16>(net, B, in, wt, bias, nullptr, nullptr, sms, s, fo, 8);
}

// Reads back (and clears) the tcgen05 convolutions' failure flag: SQ_ETIMEOUT
// if a bounded wait gave up since the last check. Synchronizes `s`.
int check_conv_err(sq_net *net, cudaStream_t s) {
  SQN_CK(cudaMemcpyAsync(net->h_err, net->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SQN_CK(cudaMemsetAsync(net->d_err, 0, sizeof(int), s));
  SQN_CK(cudaStreamSynchronize(s));
  return *net->h_err ? SQ_ETIMEOUT : SQ_OK;
}

int pack_all(sq_net *net, cudaStream_t s) {
  for (int l = 1; l < kLayers; ++l) {
    const int coutp = (l == kLayers - 1) ? 8 : kC;
    const int coutp2 = (l == kLayers - 1) ? 16 : kC;
    const int n = 27 * std::max(coutp * net->cin[l], net->cin[l] * coutp2);
    k_pack_weights<<<(n + 255) / 256, 256, 0, s>>>(net->d_w + net->woff[l], net->cout[l], net->cin[l], coutp,
                                                   net->d_wf[l], net->d_wb[l], coutp2);
    SQN_CK(cudaGetLastError());
  }
  return SQ_OK;
}

int forward(sq_net *net, int B, cudaStream_t s) {
  const int N = net->N;
  const long long N3 = (long long)N * N * N, tot = (long long)B * N3;
  k_conv_in<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(net->d_f, net->d_w + net->woff[0], net->d_w + net->boff[0],
                                                          net->d_z[0], net->d_a[0], N, tot);
  SQN_CK(cudaGetLastError());
  int st;
  for (int l = 1; l < 5; ++l) {
    st = conv32<EPI_GELU>(net, B, net->d_a[l - 1], net->d_wf[l], net->d_w + net->boff[l], net->d_z[l], net->d_a[l],
                          s);
    if (st != SQ_OK) return st;
  }
  return conv_out(net, B, net->d_a[4], net->d_wf[5], net->d_w + net->boff[5], net->d_y, s);
}

template <int CA, int CG>
int weight_grad(sq_net *net, int B, const void *A, const __nv_bfloat16 *G, int CGS, int layer, cudaStream_t s) {
  const int N = net->N;
  const long long tot = (long long)B * N * N * N;
  const int nchunk = (int)((tot + net->chunk - 1) / net->chunk);
  if (nchunk > net->nchunk) return SQ_EINVAL;
  if constexpr (CA == 32) {
    // taps on the tensor cores, the bias (tap 27) by a plain reduction
    constexpr int CGM = CG > 16 ? 32 : 16;
    const size_t smem = ((size_t)4 * N * (CGM + 8) + (size_t)6 * N * 40) * sizeof(__nv_bfloat16);
    auto kern = k_dw_mma<CGM>;
    SQN_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<dim3(nchunk, 3), 256, smem, s>>>(reinterpret_cast<const __nv_bfloat16 *>(A), G, CGS, CG, N, tot,
                                            net->chunk, net->d_dwpart);
    SQN_CK(cudaGetLastError());
    k_db<<<nchunk, 256, 0, s>>>(G, CGS, CG, tot, net->chunk, CG * CA, CA, net->d_dwpart);
  } else {
    static_assert(CA == 1 && CG == 32, "layer 1: one input channel, 32 output channels");
    k_dw_in<<<nchunk, 256, 0, s>>>(reinterpret_cast<const float *>(A), G, N, tot, net->chunk, net->d_dwpart);
  }
  SQN_CK(cudaGetLastError());
  const int nout = CG * CA;
  k_dw_reduce<<<(28 * nout + 255) / 256, 256, 0, s>>>(net->d_dwpart, nchunk, nout, CA, net->d_g + net->woff[layer],
                                                      net->d_g + net->boff[layer]);
  SQN_CK(cudaGetLastError());
  return SQ_OK;
}

int backward(sq_net *net, int B, cudaStream_t s) {
  const int N = net->N;
  const long long N3 = (long long)N * N * N;
  const long long n8 = (long long)B * N3 * kC / 8;
  int st;
  // layer 6 (32 -> 3): weights from a5 and g6, data gradient g6 -> ga
  if ((st = weight_grad<32, 3>(net, B, net->d_a[4], net->d_g6, 16, 5, s)) != SQ_OK) return st;
  if ((st = conv<16, 16, 32, EPI_PLAIN>(net, B, net->d_g6, net->d_wb[5], nullptr, nullptr, net->d_ga, nullptr, s)) !=
      SQ_OK)
    return st;
  // layers 5..2 (32 -> 32)
  for (int l = 4; l >= 1; --l) {
    k_gelu_bwd<<<(unsigned)((n8 + 255) / 256), 256, 0, s>>>(net->d_ga, net->d_z[l], net->d_gz, n8);
    SQN_CK(cudaGetLastError());
    if ((st = weight_grad<32, 32>(net, B, net->d_a[l - 1], net->d_gz, 32, l, s)) != SQ_OK) return st;
    if ((st = conv32<EPI_PLAIN>(net, B, net->d_gz, net->d_wb[l], nullptr, nullptr, net->d_ga, s)) != SQ_OK)
      return st;
  }
  // layer 1 (1 -> 32): weights only
  k_gelu_bwd<<<(unsigned)((n8 + 255) / 256), 256, 0, s>>>(net->d_ga, net->d_z[0], net->d_gz, n8);
  SQN_CK(cudaGetLastError());
  return weight_grad<1, 32>(net, B, net->d_f, net->d_gz, 32, 0, s);
}

// SplitMix64-driven normal draws (Box-Muller) for the initial weights.
struct HostRng {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(6.283185307179586 * uniform()); }
};

template <typename T>
T *nalloc(sq_net *net, size_t count, bool *ok) {
  void *p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    *ok = false;
    return nullptr;
  }
  net->allocs.push_back(p);
  return static_cast<T *>(p);
}

int feature_all(sq_net *net, int B, const sq_coeffs *const *cs, cudaStream_t s) {
  const long long N3 = (long long)net->N * net->N * net->N;
  for (int b = 0; b < B; ++b) {
    CellsDev c;
    if (coeffs_view(cs[b], &c) != SQ_OK || c.N != net->N) return SQ_EINVAL;
    k_feature<<<(unsigned)((N3 + 255) / 256), 256, 0, s>>>(c.phase, c.L, c.n, c.sub_lo, c.sub_hi,
                                                            net->d_f + b * N3);
    SQN_CK(cudaGetLastError());
  }
  return SQ_OK;
}

}  // namespace

namespace sq {
int set_conv_tc(int on) {
  if (on != 0 && on != 1 && on != 2 && on != 4) return 1;
  g_conv_tc = on;
  return 0;
}
}  // namespace sq

extern "C" {

int sq_net_create(int N, int max_batch, uint64_t seed, double out_scale, sq_net **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (N < 32 || N > 128 || N % 32 != 0 || max_batch < 1 || max_batch > 64 || !(out_scale > 0.0)) return SQ_EINVAL;
  sq_net *net = new (std::nothrow) sq_net();
  if (!net) return SQ_ENOMEM;
  net->N = N;
  net->max_batch = max_batch;
  net->out_scale = out_scale;
  long long off = 0;
  for (int l = 0; l < kLayers; ++l) {
    net->cin[l] = (l == 0) ? 1 : kC;
    net->cout[l] = (l == kLayers - 1) ? 3 : kC;
    net->woff[l] = off;
    off += 27LL * net->cin[l] * net->cout[l];
    net->boff[l] = off;
    off += net->cout[l];
  }
  net->nparam = off;
  const size_t N3 = (size_t)N * N * N, BN = N3 * max_batch;
  bool ok = true;
  net->d_w = nalloc<float>(net, off, &ok);
  net->d_g = nalloc<float>(net, off, &ok);
  net->d_m = nalloc<float>(net, off, &ok);
  net->d_v = nalloc<float>(net, off, &ok);
  for (int l = 1; l < kLayers; ++l) {
    const int coutp = (l == kLayers - 1) ? 8 : kC, coutp2 = (l == kLayers - 1) ? 16 : kC;
    net->d_wf[l] = nalloc<__nv_bfloat16>(net, 27 * coutp * net->cin[l], &ok);
    net->d_wb[l] = nalloc<__nv_bfloat16>(net, 27 * net->cin[l] * coutp2, &ok);
  }
  net->d_f = nalloc<float>(net, BN, &ok);
  net->d_y = nalloc<float>(net, 3 * BN, &ok);
  net->d_t = nalloc<float>(net, 3 * BN, &ok);
  for (int l = 0; l < 5; ++l) {
    net->d_z[l] = nalloc<__nv_bfloat16>(net, BN * kC, &ok);
    net->d_a[l] = nalloc<__nv_bfloat16>(net, BN * kC, &ok);
  }
  net->d_g6 = nalloc<__nv_bfloat16>(net, BN * 16, &ok);
  net->d_ga = nalloc<__nv_bfloat16>(net, BN * kC, &ok);
  net->d_gz = nalloc<__nv_bfloat16>(net, BN * kC, &ok);
  // about 8192 voxels, a multiple of 4 N: the tensor-core weight gradient
  // stages whole 4-row tiles of one plane (N^2 is a multiple of 4 N, so a tile
  // never crosses a plane, and B N^3 is one too, so the last tile ends at the
  // last voxel)
  net->chunk = 4 * N * std::max(1, 8192 / (4 * N));
  net->nchunk = (int)((BN + net->chunk - 1) / net->chunk);
  net->d_dwpart = nalloc<float>(net, (size_t)net->nchunk * 28 * kC * kC, &ok);
  net->d_e = nalloc<float>(net, 3 * BN, &ok);
  net->d_ae = nalloc<float>(net, 3 * BN, &ok);
  net->d_st = nalloc<Scalars>(net, 1, &ok);
  net->d_partials = nalloc<double>(net, (size_t)kMaxQ * kMaxPartials, &ok);
  const int lblocks = (int)((3 * BN + 255) / 256);
  net->d_lpart = nalloc<double>(net, lblocks, &ok);
  if (ok && cudaMallocHost(&net->h_lpart, sizeof(double) * lblocks) != cudaSuccess) ok = false;
  net->d_err = nalloc<int>(net, 1, &ok);
  if (ok && cudaMallocHost(&net->h_err, sizeof(int)) != cudaSuccess) ok = false;
  if (ok && cudaMemset(net->d_err, 0, sizeof(int)) != cudaSuccess) ok = false;
  if (ok && cudaMemset(net->d_st, 0, sizeof(Scalars)) != cudaSuccess) ok = false;
  if (!ok) {
    sq_net_destroy(net);
    return SQ_ENOMEM;
  }
  // He-normal weights (last layer scaled down so the first guess is near zero), zero biases
  std::vector<float> w(off, 0.f);
  HostRng rng{seed};
  for (int l = 0; l < kLayers; ++l) {
    const double sd = std::sqrt(2.0 / (27.0 * net->cin[l])) * ((l == kLayers - 1) ? 0.1 : 1.0);
    for (long long i = 0; i < 27LL * net->cin[l] * net->cout[l]; ++i) w[net->woff[l] + i] = (float)(sd * rng.normal());
  }
  if (sq_net_set_params(net, w.data(), off) != SQ_OK) {
    sq_net_destroy(net);
    return SQ_ECUDA;
  }
  *out = net;
  return SQ_OK;
}

void sq_net_destroy(sq_net *net) {
  if (!net) return;
  for (void *p : net->allocs) cudaFree(p);
  if (net->h_lpart) cudaFreeHost(net->h_lpart);
  if (net->h_err) cudaFreeHost(net->h_err);
  delete net;
}

int sq_net_params(const sq_net *net, float *host, int64_t *count) {
  if (!net) return SQ_EINVAL;
  if (count) *count = net->nparam;
  if (host) SQN_CK(cudaMemcpy(host, net->d_w, sizeof(float) * net->nparam, cudaMemcpyDeviceToHost));
  return SQ_OK;
}

int sq_net_grads(const sq_net *net, float *host, int64_t count) {
  if (!net || !host || count != net->nparam) return SQ_EINVAL;
  SQN_CK(cudaMemcpy(host, net->d_g, sizeof(float) * count, cudaMemcpyDeviceToHost));
  return SQ_OK;
}

int sq_net_set_params(sq_net *net, const float *host, int64_t count) {
  if (!net || !host || count != net->nparam) return SQ_EINVAL;
  SQN_CK(cudaMemcpy(net->d_w, host, sizeof(float) * count, cudaMemcpyHostToDevice));
  SQN_CK(cudaMemset(net->d_m, 0, sizeof(float) * count));
  SQN_CK(cudaMemset(net->d_v, 0, sizeof(float) * count));
  net->step = 0;
  int st = pack_all(net, 0);
  if (st != SQ_OK) return st;
  SQN_CK(cudaDeviceSynchronize());
  return SQ_OK;
}

int sq_net_predict(sq_net *net, const sq_coeffs *c, double *psi0, double *psi1, double *psi2, sq_stream_t stream) {
  if (!net || !c || !psi0 || !psi1 || !psi2) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = feature_all(net, 1, &c, s);
  if (st != SQ_OK) return st;
  if ((st = forward(net, 1, s)) != SQ_OK) return st;
  const long long N3 = (long long)net->N * net->N * net->N;
  k_to_psi<<<(unsigned)((N3 + 255) / 256), 256, 0, s>>>(net->d_y, psi0, psi1, psi2, N3);
  SQN_CK(cudaGetLastError());
  return g_conv_tc ? check_conv_err(net, s) : SQ_OK;
}

int sq_net_train_step(sq_net *net, int batch, const sq_coeffs *const *cs, const double *const *targets, float lr,
                      int loss_type, double *loss, sq_stream_t stream) {
  if (!net || !cs || !targets || batch < 1 || batch > net->max_batch || !(lr > 0.f) || loss_type < 0 ||
      loss_type > 2)
    return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long N3 = (long long)net->N * net->N * net->N;
  int st = feature_all(net, batch, cs, s);
  if (st != SQ_OK) return st;
  for (int b = 0; b < batch; ++b) {
    if (!targets[3 * b] || !targets[3 * b + 1] || !targets[3 * b + 2]) return SQ_EINVAL;
    k_target_f32<<<(unsigned)((N3 + 255) / 256), 256, 0, s>>>(targets[3 * b], targets[3 * b + 1],
                                                              targets[3 * b + 2], net->d_t + 3 * b * N3, N3);
    SQN_CK(cudaGetLastError());
  }
  if ((st = forward(net, batch, s)) != SQ_OK) return st;
  const long long tot = (long long)batch * N3;
  int lblocks;
  if (loss_type == 0) {
    // mean squared error of (y - t) / out_scale
    lblocks = (int)((tot + 255) / 256);
    k_loss_grad<<<lblocks, 256, 0, s>>>(net->d_y, net->d_t, net->d_g6, (float)(1.0 / net->out_scale),
                                        net->d_lpart, N3, batch);
    SQN_CK(cudaGetLastError());
  } else if (loss_type == 2) {
    // residual norm of the guess: L = sum_i r_i . r_i, r = (A y - b_i) / out_scale
    // (the norm the solver's stopping rule measures; no targets needed), with
    // dL/d(conv6 out) = 2 A r (A is symmetric)
    const long long n = 3 * tot;
    RedBuf rb;
    rb.st = net->d_st;
    rb.partials = net->d_partials;
    for (int b = 0; b < batch; ++b) {
      CellsDev c;
      if (coeffs_view(cs[b], &c) != SQ_OK) return SQ_EINVAL;
      for (int i = 0; i < 3; ++i) {
        const long long o = (3LL * b + i) * N3;
        SQN_CK((launch_stencil<float, float>(c, ST_MATVEC, 0, net->d_y + o, net->d_ae + o, rb, FIN_NONE, false, s)));
        SQN_CK((launch_stencil<double, float>(c, ST_RHS, i, nullptr, net->d_e + o, rb, FIN_NONE, false, s)));
      }
    }
    k_sub_scale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(net->d_ae, net->d_e, (float)(1.0 / net->out_scale), n);
    SQN_CK(cudaGetLastError());
    for (int b = 0; b < batch; ++b) {
      CellsDev c;
      if (coeffs_view(cs[b], &c) != SQ_OK) return SQ_EINVAL;
      for (int i = 0; i < 3; ++i) {
        const long long o = (3LL * b + i) * N3;
        SQN_CK((launch_stencil<float, float>(c, ST_MATVEC, 0, net->d_e + o, net->d_ae + o, rb, FIN_NONE, false, s)));
      }
    }
    lblocks = (int)((n + 255) / 256);
    k_dot_partial<<<lblocks, 256, 0, s>>>(net->d_e, net->d_e, net->d_lpart, n);
    k_pack_grad<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(net->d_ae, net->d_g6, N3, batch);
    SQN_CK(cudaGetLastError());
  } else {
    // energy norm of the error: L = sum_i e_i . A e_i, e = (y - t) / out_scale,
    // with the operator of each sample's realization (FP32 stencil kernel)
    const long long n = 3 * tot;
    k_err<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(net->d_y, net->d_t, net->d_e, (float)(1.0 / net->out_scale), n);
    SQN_CK(cudaGetLastError());
    RedBuf rb;
    rb.st = net->d_st;
    rb.partials = net->d_partials;
    for (int b = 0; b < batch; ++b) {
      CellsDev c;
      if (coeffs_view(cs[b], &c) != SQ_OK) return SQ_EINVAL;
      for (int i = 0; i < 3; ++i) {
        const long long o = (3LL * b + i) * N3;
        SQN_CK((launch_stencil<float, float>(c, ST_MATVEC, 0, net->d_e + o, net->d_ae + o, rb, FIN_NONE, false, s)));
      }
    }
    lblocks = (int)((n + 255) / 256);
    k_dot_partial<<<lblocks, 256, 0, s>>>(net->d_e, net->d_ae, net->d_lpart, n);
    k_pack_grad<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(net->d_ae, net->d_g6, N3, batch);
    SQN_CK(cudaGetLastError());
  }
  if ((st = backward(net, batch, s)) != SQ_OK) return st;
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
  k_adam<<<(unsigned)((net->nparam + 255) / 256), 256, 0, s>>>(net->d_w, net->d_g, net->d_m, net->d_v,
                                                               (int)net->nparam, lr, b1, b2, 1e-8f, c1, c2);
  SQN_CK(cudaGetLastError());
  if ((st = pack_all(net, s)) != SQ_OK) return st;
  if (loss) {
    SQN_CK(cudaMemcpyAsync(net->h_lpart, net->d_lpart, sizeof(double) * lblocks, cudaMemcpyDeviceToHost, s));
    SQN_CK(cudaStreamSynchronize(s));
    double t = 0.0;
    for (int i = 0; i < lblocks; ++i) t += net->h_lpart[i];
    *loss = t / (3.0 * (double)tot);
    if (g_conv_tc) return check_conv_err(net, s);
  }
  return SQ_OK;
}

}  // extern "C"
