// Device core of the matrix-free operator, shared by the single-solve and the
// batched kernels. See stencil.cu for the operator and its edge coefficients.
#pragma once

#include "common.cuh"

namespace sq {

// ------------------------------------------------------ coefficient patterns
// Bit s1*4 + s2*2 + s3 of the pattern = phase of voxel (j1-s1, j2-s2, j3-s3).
// Entries: 0 a_1(j), 1 a_1(j-e1), 2 a_2(j), 3 a_2(j-e2), 4 a_3(j), 5 a_3(j-e3),
// 6 diagonal (sum of the six), 7.. unused (odd row stride: no bank conflicts
// between nodes that see different patterns). Multi-level media keep one
// 256-row table per threshold layer (rows l*256 + pattern; see CellsDev): the
// pattern of layer l has the bit "voxel level >= l + 1" and the node's
// coefficients are the sum of its layers' rows.
constexpr int kTabStride = 9;
template <typename T>
__device__ __forceinline__ void build_pattern_table(T (*tab)[kTabStride], const CellsDev &c, int tid) {
  const unsigned face[6] = {0x0Fu, 0xF0u, 0x33u, 0xCCu, 0x55u, 0xAAu};
  for (int row = tid; row < 256 * c.layers; row += kThreads) {
    const int l = row >> 8, m = row & 255;
    const T *ev = edge_table<T>(c, l);
    const T *dv = diag_table<T>(c, l);
    int kk = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int k = __popc(m & face[f]);
      tab[row][f] = ev[k];
      kk += k;
    }
    tab[row][6] = dv[kk];
    for (int f = 7; f < kTabStride; ++f) tab[row][f] = (T)0;
  }
}

// Layer bits of one phase byte v: bit 8l set iff v >= l + 1 (layers 0..2).
// The plain checkerboard kernels (ML = false, compiled without the extra
// layers) read only bit 0, i.e. any nonzero phase is high.
template <bool ML = true>
__device__ __forceinline__ unsigned level_bits(unsigned v) {
  if constexpr (ML)
    return (v != 0u ? 1u : 0u) | (v >= 2u ? 0x100u : 0u) | (v >= 3u ? 0x10000u : 0u);
  else
    return v != 0u ? 1u : 0u;
}
// Replicates a mask of layer-0 bits into every layer's byte.
__device__ __forceinline__ unsigned all_layers(unsigned m) { return m * 0x10101u; }

// Four phase bits of cell row c1 at the node's (s2, s3) cell offsets, one
// nibble per layer (bits 8l .. 8l+3).
__device__ __forceinline__ unsigned load4(const uint8_t *__restrict__ phase, int c1, int LL, int o00, int o01,
                                          int o10, int o11) {
  const uint8_t *ph = phase + (size_t)c1 * LL;
  return level_bits(ph[o00]) | (level_bits(ph[o01]) << 1) | (level_bits(ph[o10]) << 2) | (level_bits(ph[o11]) << 3);
}

// Sub-cell inclusions: can the voxel at cell-local index u (one axis) be high?
__device__ __forceinline__ bool in_sub(const CellsDev &c, int u) { return u >= c.sub_lo && u < c.sub_hi; }
// Node patterns change between planes j1 - 1 and j1 where a voxel plane
// crosses a cell face (cell position 0, 1) or a sub-cell face (sub_lo,
// sub_lo + 1, sub_hi, sub_hi + 1); for whole cells only at 0 and 1.
// GEN = false compiles the plain checkerboard (two levels, whole cells).
template <bool GEN>
__device__ __forceinline__ bool pattern_changes(const CellsDev &c, int cpos) {
  if constexpr (!GEN) return cpos <= 1;
  return cpos <= 1 || cpos == c.sub_lo || cpos == c.sub_lo + 1 || cpos == c.sub_hi || cpos == c.sub_hi + 1;
}
// Plane masks of a node at cell position cpos: the voxels of plane j1 (low
// nibble) and of plane j1 - 1 (high nibble) may be high.
template <bool GEN>
__device__ __forceinline__ void plane_masks(const CellsDev &c, int cpos, unsigned &pm0, unsigned &pm1) {
  if constexpr (!GEN) {
    pm0 = pm1 = 0xFu;
    return;
  }
  pm0 = in_sub(c, cpos) ? 0xFu : 0u;
  pm1 = in_sub(c, cpos == 0 ? c.n - 1 : cpos - 1) ? 0xFu : 0u;
}
// In-plane inclusion mask of a node row (see row_nibbles).
template <bool GEN>
__device__ __forceinline__ unsigned row_mask(const CellsDev &c, int u2, unsigned m3) {
  if constexpr (!GEN) return 0x3u;
  return in_sub(c, u2) ? m3 : 0u;
}

// ------------------------------------------------------------ stencil kernel
// A thread owns RPT consecutive node rows j2b .. j2b+RPT-1 of column j3 and
// marches along j1 over [z0, z1). Per row it keeps x(j1-1), x(j1) in
// registers and the next kAhead planes' values in a register queue; the
// march is unrolled by kAhead so that queue slot u is consumed and refilled
// in place at step u of every round (the load of plane j1+1+kAhead is issued
// kAhead steps before its use and no register waits on a load in flight
// before then). The j2-neighbours inside the row group are the other rows'
// x(j1) registers; rows j2b-1 and j2b+RPT and the j3-neighbours are loaded
// (L1/L2 hits: neighbouring threads loaded them as queue entries). Planes
// past z1 are never loaded.
// Coefficients: the eight voxel bits of a node, and with them its seven
// coefficients (held in registers), change only at the planes j1 = 0, 1
// (mod n); j1 is the same for the whole block there, so the reload branch is
// uniform. `cellof` is a shared-memory table j -> j / n of the block.
// Pattern nibbles of the RPT rows for cell plane c1: bit 0 / 1 = the row's
// own cell at j3 / j3-1, bit 2 / 3 = the cell of row j2-1 at j3 / j3-1.
// crow[q] = (cell of row j2b-1+q) * L.
// mq[q]: in-plane inclusion mask of row q (bits 0 / 1: the voxel at j3 / j3-1
// of that row may be high; the same bits in every layer's byte).
template <int RPT, bool ML>
__device__ __forceinline__ void row_nibbles(const uint8_t *__restrict__ phase, int c1, int LL, const int (&crow)[RPT + 1],
                                            int c3a, int c3b, const unsigned (&mq)[RPT + 1], unsigned (&nb)[RPT]) {
  const uint8_t *ph = phase + (size_t)c1 * LL;
  unsigned b[RPT + 1];
#pragma unroll
  for (int q = 0; q <= RPT; ++q)
    b[q] = (level_bits<ML>(ph[crow[q] + c3a]) | (level_bits<ML>(ph[crow[q] + c3b]) << 1)) & mq[q];
#pragma unroll
  for (int r = 0; r < RPT; ++r) nb[r] = b[r + 1] | (b[r] << 2);
}

// Coefficients of the RPT rows from their current (nc) and previous-plane
// (np) nibbles: layer 0's table row, plus the higher layers' rows for
// multi-level media (block-uniform branch on c.layers).
template <typename Ti, int RPT, bool ML>
__device__ __forceinline__ void row_coeffs(const Ti (*tab)[kTabStride], int layers, const unsigned (&nc)[RPT],
                                           const unsigned (&np)[RPT], unsigned pm0, unsigned pm1, Ti (&t)[RPT][7]) {
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const Ti *tr = tab[(nc[r] & pm0) | ((np[r] & pm1) << 4)];
#pragma unroll
    for (int k = 0; k < 7; ++k) t[r][k] = tr[k];
  }
  if constexpr (!ML) return;
#pragma unroll
  for (int l = 1; l < kMaxLayers; ++l) {
    if (l < layers) {
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const Ti *tr = tab[256 * l + ((((nc[r] >> (8 * l)) & pm0)) | (((np[r] >> (8 * l)) & pm1) << 4))];
#pragma unroll
        for (int k = 0; k < 7; ++k) t[r][k] += tr[k];
      }
    }
  }
}

// Fills cellof[j] = j / n for j < N (block-cooperative; caller syncs).
__device__ __forceinline__ void build_cellof(short *cellof, int N, int n, int tid) {
  for (int j = tid; j < N; j += kThreads) cellof[j] = (short)(j / n);
}

template <typename Ti, typename To, int MODE, int RPT, bool GEN, int kAhead = 4>
__device__ __forceinline__ void stencil_rows(const CellsDev &c, int dir, const Ti *__restrict__ x, To *__restrict__ y,
                                             const Ti (*tab)[kTabStride], const short *__restrict__ cellof, int j3,
                                             int j2b, int z0, int z1, Accum<Ti> &acc0, Accum<Ti> &acc1) {
  const int N = c.N, n = c.n, L = c.L;
  const int NN = N * N;  // N^3 < 2^31 for N <= 512: int indices
  const int LL = L * L;
  const int j3m = (j3 == 0) ? N - 1 : j3 - 1, j3p = (j3 == N - 1) ? 0 : j3 + 1;
  const int c3a = cellof[j3], c3b = cellof[j3m];
  const int d3p = j3p - j3, d3m = j3m - j3;
  int crow[RPT + 1];
  unsigned mq[RPT + 1];  // in-plane inclusion masks (see row_nibbles)
  const unsigned m3 = all_layers((in_sub(c, j3 - c3a * n) ? 1u : 0u) | (in_sub(c, j3m - c3b * n) ? 2u : 0u));
#pragma unroll
  for (int q = 0; q <= RPT; ++q) {
    const int j2 = (j2b - 1 + q < 0) ? N - 1 : j2b - 1 + q;  // rows j2b .. j2b+RPT-1 are < N
    crow[q] = cellof[j2] * L;
    mq[q] = row_mask<GEN>(c, j2 - cellof[j2] * n, m3);
  }
  const int row0 = j2b * N + j3;
  const int up = ((j2b == 0) ? N - 1 : j2b - 1) * N + j3 - row0;          // row j2b - 1
  const int dn = ((j2b + RPT >= N) ? j2b + RPT - N : j2b + RPT) * N + j3 - row0;  // row j2b + RPT

  const int j1m0 = (z0 == 0) ? N - 1 : z0 - 1;
  int cpos = z0 - cellof[z0] * n;  // position of plane z0 within its cell
  unsigned np[RPT], nc[RPT], pm0, pm1;
  row_nibbles<RPT, GEN>(c.phase, cellof[j1m0], LL, crow, c3a, c3b, mq, np);
  if (cpos == 0) {
    row_nibbles<RPT, GEN>(c.phase, cellof[z0], LL, crow, c3a, c3b, mq, nc);
  } else {
#pragma unroll
    for (int r = 0; r < RPT; ++r) nc[r] = np[r];
  }
  plane_masks<GEN>(c, cpos, pm0, pm1);
  Ti t[RPT][7];
  row_coeffs<Ti, RPT, GEN>(tab, c.layers, nc, np, pm0, pm1, t);

  Ti xm[RPT], x0[RPT], ahead[RPT][kAhead];  // ahead[r][u] = x(jb + 1 + u) of row r
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    xm[r] = x0[r] = (Ti)0;
#pragma unroll
    for (int u = 0; u < kAhead; ++u) ahead[r][u] = (Ti)0;
  }
  if (MODE != ST_RHS) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      xm[r] = x[j1m0 * NN + row0 + r * N];
      x0[r] = x[z0 * NN + row0 + r * N];
    }
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      const int jj = z0 + 1 + u;
      if (jj <= z1) {
        const int pl = (jj >= N ? jj - N : jj) * NN + row0;
#pragma unroll
        for (int r = 0; r < RPT; ++r) ahead[r][u] = x[pl + r * N];
      }
    }
  }
  for (int jb = z0; jb < z1; jb += kAhead) {
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      const int j1 = jb + u;
      if (j1 < z1) {
        if (j1 > z0) {
          cpos = (cpos + 1 == n) ? 0 : cpos + 1;
          if (pattern_changes<GEN>(c, cpos)) {
            if (cpos <= 1) {
#pragma unroll
              for (int r = 0; r < RPT; ++r) np[r] = nc[r];
            }
            if (cpos == 0) row_nibbles<RPT, GEN>(c.phase, cellof[j1], LL, crow, c3a, c3b, mq, nc);
            plane_masks<GEN>(c, cpos, pm0, pm1);
            row_coeffs<Ti, RPT, GEN>(tab, c.layers, nc, np, pm0, pm1, t);
          }
        }
        const int b0 = j1 * NN + row0;
        Ti xp[RPT];
        if (MODE != ST_RHS) {
#pragma unroll
          for (int r = 0; r < RPT; ++r) xp[r] = ahead[r][u];
          const int jj = j1 + 1 + kAhead;
          if (jj <= z1) {
            const int pl = (jj >= N ? jj - N : jj) * NN + row0;
#pragma unroll
            for (int r = 0; r < RPT; ++r) ahead[r][u] = x[pl + r * N];
          }
        }
        Ti psum = (Ti)0;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const int idx = b0 + r * N;
          Ti out;
          Ti bv = (Ti)0;
          if (MODE != ST_MATVEC) bv = (dir == 0) ? t[r][0] - t[r][1] : (dir == 1) ? t[r][2] - t[r][3] : t[r][4] - t[r][5];
          if (MODE != ST_RHS) {
            const Ti x2m = (r == 0) ? x[b0 + up] : x0[r > 0 ? r - 1 : 0];
            const Ti x2p = (r == RPT - 1) ? x[b0 + dn] : x0[r + 1 < RPT ? r + 1 : r];
            const Ti x3p = x[idx + d3p], x3m = x[idx + d3m];
            Ti off = t[r][0] * xp[r];
            off = fma(t[r][1], xm[r], off);
            off = fma(t[r][2], x2p, off);
            off = fma(t[r][3], x2m, off);
            off = fma(t[r][4], x3p, off);
            off = fma(t[r][5], x3m, off);
            const Ti ax = fma(t[r][6], x0[r], -off);
            if (MODE == ST_MATVEC) {
              out = ax;
              if (RPT == 1)
                acc0.add_prod(x0[r], ax);
              else
                psum = fma(x0[r], ax, psum);
            } else {
              out = bv - ax;
              acc0.add_prod(out, out);
              acc1.add_prod(bv, bv);
            }
          } else {
            out = bv;
            acc0.add_prod(bv, bv);
            acc1.add_prod(bv, bv);
          }
          y[idx] = (To)out;
        }
        if (MODE == ST_MATVEC && RPT > 1) acc0.add(psum);
        if (MODE != ST_RHS) {
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            xm[r] = x0[r];
            x0[r] = xp[r];
          }
        }
      }
    }
  }
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

__device__ __forceinline__ void cp_async16(unsigned dst, const float *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(unsigned dst, const float *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// A thread's share of copying one plane of the tile (j2_0, j3_0) with its
// halo: a 16-byte body chunk, and for threads 0..15 a 16-byte halo-row chunk
// or for threads 16..79 one halo-column float. The in-plane source offsets and
// the slot offsets are fixed per thread and computed once.
struct PlaneCopy {
  int src0, dst0;  // body chunk: element offset in a plane, byte offset in a slot
  int src1, dst1;  // halo element, or -1
  int wide1;       // halo is a 16-byte chunk (1) or one float (0)
  __device__ __forceinline__ void init(int N, int j2_0, int j3_0, int tid) {
    const int row = tid >> 3, ch = tid & 7;
    src0 = (j2_0 + row) * N + j3_0 + 4 * ch;
    dst0 = ((1 + row) * kSW + 4 + 4 * ch) * 4;
    src1 = -1;
    dst1 = 0;
    wide1 = 0;
    if (tid < 16) {  // halo rows j2_0 - 1 and j2_0 + 32
      const int hr = tid >> 3;
      const int gr = hr ? (j2_0 + 32 == N ? 0 : j2_0 + 32) : (j2_0 == 0 ? N - 1 : j2_0 - 1);
      src1 = gr * N + j3_0 + 4 * ch;
      dst1 = ((hr ? kSRows - 1 : 0) * kSW + 4 + 4 * ch) * 4;
      wide1 = 1;
    } else if (tid < 80) {  // halo columns j3_0 - 1 and j3_0 + 32
      const int e = tid - 16, side = e >> 5, hrow = e & 31;
      const int gc = side ? (j3_0 + 32 == N ? 0 : j3_0 + 32) : (j3_0 == 0 ? N - 1 : j3_0 - 1);
      src1 = (j2_0 + hrow) * N + gc;
      dst1 = ((1 + hrow) * kSW + (side ? 36 : 3)) * 4;
    }
  }
  // Issues the copies of plane `pl` (the plane's first element) into the slot
  // at shared address `slot`.
  __device__ __forceinline__ void issue(const float *pl, unsigned slot) const {
    cp_async16(slot + dst0, pl + src0);
    if (src1 >= 0) {
      if (wide1)
        cp_async16(slot + dst1, pl + src1);
      else
        cp_async4(slot + dst1, pl + src1);
    }
  }
};

// Runs the staged FP32 operator y = A x (MATVEC) over planes [z0, z1) of the
// 32 x 32 tile (j2_0, j3_0) and adds p.Ap to acc. Builds the block's pattern
// and cell tables itself; `ring` is kStages * kSlot floats of 16-byte aligned
// shared memory. All threads of the block (32 x 8) must call it.
template <bool GEN>
__device__ __forceinline__ void stencil_staged_run(const CellsDev &c, const float *__restrict__ x,
                                                   float *__restrict__ y, float (*tab)[kTabStride], short *cellof,
                                                   float *ring, int j2_0, int j3_0, int z0, int z1,
                                                   Accum<float> &acc) {
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const int N = c.N, n = c.n, L = c.L, LL = L * L;
  const int NN = N * N;
  PlaneCopy cp;
  cp.init(N, j2_0, j3_0, tid);
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  const size_t plane = (size_t)NN;
  // prologue: planes z0 .. z0 + kStages - 2 (one commit group each, empty past z1)
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    const int j = z0 + st;
    if (j <= z1) cp.issue(x + (j == N ? 0 : (size_t)j * plane), ring_s + st * kSlot * 4);
    cp_async_commit();
  }
  __syncthreads();  // the caller's previous use of the tables is over
  build_pattern_table<float>(tab, c, tid);
  build_cellof(cellof, N, n, tid);
  __syncthreads();

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j3 = j3_0 + tx, j2b = j2_0 + 4 * ty;
  const int j3m = (j3 == 0) ? N - 1 : j3 - 1;
  const int c3a = cellof[j3], c3b = cellof[j3m];
  int crow[5];
  unsigned mq[5];  // in-plane inclusion masks (see row_nibbles)
  const unsigned m3 = all_layers((in_sub(c, j3 - c3a * n) ? 1u : 0u) | (in_sub(c, j3m - c3b * n) ? 2u : 0u));
#pragma unroll
  for (int q = 0; q <= 4; ++q) {
    const int j2 = (j2b - 1 + q < 0) ? N - 1 : j2b - 1 + q;
    crow[q] = cellof[j2] * L;
    mq[q] = row_mask<GEN>(c, j2 - cellof[j2] * n, m3);
  }
  const int j1m0 = (z0 == 0) ? N - 1 : z0 - 1;
  int cpos = z0 - cellof[z0] * n;
  unsigned np[4], nc[4], pm0, pm1;
  row_nibbles<4, GEN>(c.phase, cellof[j1m0], LL, crow, c3a, c3b, mq, np);
  if (cpos == 0) {
    row_nibbles<4, GEN>(c.phase, cellof[z0], LL, crow, c3a, c3b, mq, nc);
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) nc[r] = np[r];
  }
  plane_masks<GEN>(c, cpos, pm0, pm1);
  float t[4][7];
  row_coeffs<float, 4, GEN>(tab, c.layers, nc, np, pm0, pm1, t);
  const int row0 = j2b * N + j3;
  float xm[4], x0[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) xm[r] = x[(size_t)j1m0 * NN + row0 + r * N];

  // The march is unrolled by the ring depth: plane j1 = z0 + k sits in slot
  // u = k mod kStages, so the slots of planes j1 (s0), j1 + 1 (s1) and
  // j1 + kStages - 1 (sr, the slot of j1 - 1) are compile-time constants.
  const int toff = (1 + 4 * ty) * kSW + 4 + tx;
  for (int kb = 0; z0 + kb < z1; kb += kStages) {
#pragma unroll
    for (int u = 0; u < kStages; ++u) {
      const int k = kb + u;
      const int j1 = z0 + k;
      if (j1 >= z1) break;
      const int s0 = u, s1 = (u + 1) % kStages, sr = (u + kStages - 1) % kStages;
      cp_async_wait<kStages - 3>();  // this thread's copies of planes j1, j1 + 1 have landed
      __syncthreads();               // ... everyone's; and everyone is done with plane j1 - 1's slot
      {
        const int j = j1 + kStages - 1;
        if (j <= z1) cp.issue(x + (size_t)(j == N ? 0 : j) * plane, ring_s + sr * kSlot * 4);
        cp_async_commit();
      }
      if (k > 0) {
        cpos = (cpos + 1 == n) ? 0 : cpos + 1;
        if (pattern_changes<GEN>(c, cpos)) {
          if (cpos <= 1) {
#pragma unroll
            for (int r = 0; r < 4; ++r) np[r] = nc[r];
          }
          if (cpos == 0) row_nibbles<4, GEN>(c.phase, cellof[j1], LL, crow, c3a, c3b, mq, nc);
          plane_masks<GEN>(c, cpos, pm0, pm1);
          row_coeffs<float, 4, GEN>(tab, c.layers, nc, np, pm0, pm1, t);
        }
      }
      const float *S0 = ring + s0 * kSlot + toff;
      const float *S1 = ring + s1 * kSlot + toff;
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
  }
  cp_async_wait<0>();
}

}  // namespace sq
