// Device core of the matrix-free operator, shared by the single-solve and the
// batched kernels. See stencil.cu for the operator and its edge coefficients.
#pragma once

#include "common.cuh"

namespace sq {

// ------------------------------------------------------ coefficient patterns
// Bit s1*4 + s2*2 + s3 of the pattern = phase of voxel (j1-s1, j2-s2, j3-s3).
// Entries: 0 a_1(j), 1 a_1(j-e1), 2 a_2(j), 3 a_2(j-e2), 4 a_3(j), 5 a_3(j-e3),
// 6 diagonal (sum of the six), 7.. unused (odd row stride: no bank conflicts
// between nodes that see different patterns).
constexpr int kTabStride = 9;
template <typename T>
__device__ __forceinline__ void build_pattern_table(T (*tab)[kTabStride], const CellsDev &c, int tid) {
  const unsigned face[6] = {0x0Fu, 0xF0u, 0x33u, 0xCCu, 0x55u, 0xAAu};
  const T *ev = edge_table<T>(c);
  const T *dv = diag_table<T>(c);
  for (int m = tid; m < 256; m += kThreads) {
    int kk = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int k = __popc(m & face[f]);
      tab[m][f] = ev[k];
      kk += k;
    }
    tab[m][6] = dv[kk];
    for (int f = 7; f < kTabStride; ++f) tab[m][f] = (T)0;
  }
}

// Four phase bits of cell row c1 at the node's (s2, s3) cell offsets.
__device__ __forceinline__ unsigned load4(const uint8_t *__restrict__ phase, int c1, int LL, int o00, int o01,
                                          int o10, int o11) {
  const uint8_t *ph = phase + (size_t)c1 * LL;
  return (ph[o00] ? 1u : 0u) | (ph[o01] ? 2u : 0u) | (ph[o10] ? 4u : 0u) | (ph[o11] ? 8u : 0u);
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
template <int RPT>
__device__ __forceinline__ void row_nibbles(const uint8_t *__restrict__ phase, int c1, int LL, const int (&crow)[RPT + 1],
                                            int c3a, int c3b, unsigned (&nb)[RPT]) {
  const uint8_t *ph = phase + (size_t)c1 * LL;
  unsigned b[RPT + 1];
#pragma unroll
  for (int q = 0; q <= RPT; ++q) b[q] = (ph[crow[q] + c3a] ? 1u : 0u) | (ph[crow[q] + c3b] ? 2u : 0u);
#pragma unroll
  for (int r = 0; r < RPT; ++r) nb[r] = b[r + 1] | (b[r] << 2);
}

template <typename Ti, int RPT>
__device__ __forceinline__ void row_coeffs(const Ti (*tab)[kTabStride], const unsigned (&nc)[RPT],
                                           const unsigned (&np)[RPT], Ti (&t)[RPT][7]) {
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const Ti *tr = tab[nc[r] | (np[r] << 4)];
#pragma unroll
    for (int k = 0; k < 7; ++k) t[r][k] = tr[k];
  }
}

// Fills cellof[j] = j / n for j < N (block-cooperative; caller syncs).
__device__ __forceinline__ void build_cellof(short *cellof, int N, int n, int tid) {
  for (int j = tid; j < N; j += kThreads) cellof[j] = (short)(j / n);
}

template <typename Ti, typename To, int MODE, int RPT, int kAhead = 4>
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
#pragma unroll
  for (int q = 0; q <= RPT; ++q) {
    const int j2 = (j2b - 1 + q < 0) ? N - 1 : j2b - 1 + q;  // rows j2b .. j2b+RPT-1 are < N
    crow[q] = cellof[j2] * L;
  }
  const int row0 = j2b * N + j3;
  const int up = ((j2b == 0) ? N - 1 : j2b - 1) * N + j3 - row0;          // row j2b - 1
  const int dn = ((j2b + RPT >= N) ? j2b + RPT - N : j2b + RPT) * N + j3 - row0;  // row j2b + RPT

  const int j1m0 = (z0 == 0) ? N - 1 : z0 - 1;
  int cpos = z0 - cellof[z0] * n;  // position of plane z0 within its cell
  unsigned np[RPT], nc[RPT];
  row_nibbles<RPT>(c.phase, cellof[j1m0], LL, crow, c3a, c3b, np);
  if (cpos == 0) {
    row_nibbles<RPT>(c.phase, cellof[z0], LL, crow, c3a, c3b, nc);
  } else {
#pragma unroll
    for (int r = 0; r < RPT; ++r) nc[r] = np[r];
  }
  Ti t[RPT][7];
  row_coeffs<Ti, RPT>(tab, nc, np, t);

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
          if (cpos <= 1) {
#pragma unroll
            for (int r = 0; r < RPT; ++r) np[r] = nc[r];
            if (cpos == 0) row_nibbles<RPT>(c.phase, cellof[j1], LL, crow, c3a, c3b, nc);
            row_coeffs<Ti, RPT>(tab, nc, np, t);
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

}  // namespace sq
