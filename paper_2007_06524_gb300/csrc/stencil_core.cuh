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
// One thread owns node column (j2, j3) and marches along j1 over [z0, z1),
// keeping x(j1-1), x(j1), x(j1+1) in registers. The eight voxel bits change
// only when j1 crosses a cell boundary.
template <typename Ti, typename To, int MODE>
__device__ __forceinline__ void stencil_column(const CellsDev &c, int dir, const Ti *__restrict__ x,
                                               To *__restrict__ y, const Ti (*tab)[kTabStride], int j3, int j2,
                                               int z0, int z1, Accum<Ti> &acc0, Accum<Ti> &acc1) {
  const int N = c.N, n = c.n, L = c.L;
  const size_t NN = (size_t)N * N;
  const int j3m = (j3 == 0) ? N - 1 : j3 - 1, j3p = (j3 == N - 1) ? 0 : j3 + 1;
  const int j2m = (j2 == 0) ? N - 1 : j2 - 1, j2p = (j2 == N - 1) ? 0 : j2 + 1;
  const int c3a = j3 / n, c3b = j3m / n, c2a = j2 / n, c2b = j2m / n;
  const int o00 = c2a * L + c3a, o01 = c2a * L + c3b, o10 = c2b * L + c3a, o11 = c2b * L + c3b;
  const int LL = L * L;
  const size_t row = (size_t)j2 * N + j3;
  const size_t r2p = (size_t)j2p * N + j3, r2m = (size_t)j2m * N + j3;
  const size_t r3p = (size_t)j2 * N + j3p, r3m = (size_t)j2 * N + j3m;

  int j1 = z0;
  const int j1m0 = (j1 == 0) ? N - 1 : j1 - 1;
  unsigned m_prev = load4(c.phase, j1m0 / n, LL, o00, o01, o10, o11);
  unsigned m_cur = (j1 % n == 0) ? load4(c.phase, j1 / n, LL, o00, o01, o10, o11) : m_prev;
  Ti xm = (Ti)0, x0 = (Ti)0, xp = (Ti)0;
  if (MODE != ST_RHS) {
    xm = x[(size_t)j1m0 * NN + row];
    x0 = x[(size_t)j1 * NN + row];
  }
  for (; j1 < z1; ++j1) {
    if (j1 > z0) {
      m_prev = m_cur;
      if (j1 % n == 0) m_cur = load4(c.phase, j1 / n, LL, o00, o01, o10, o11);
    }
    const Ti *t = tab[m_cur | (m_prev << 4)];
    const size_t base = (size_t)j1 * NN;
    Ti out;
    Ti bv = (Ti)0;
    if (MODE != ST_MATVEC) bv = t[2 * dir] - t[2 * dir + 1];
    if (MODE != ST_RHS) {
      const int j1p = (j1 == N - 1) ? 0 : j1 + 1;
      xp = x[(size_t)j1p * NN + row];
      const Ti x2p = x[base + r2p], x2m = x[base + r2m];
      const Ti x3p = x[base + r3p], x3m = x[base + r3m];
      Ti off = t[0] * xp;
      off = fma(t[1], xm, off);
      off = fma(t[2], x2p, off);
      off = fma(t[3], x2m, off);
      off = fma(t[4], x3p, off);
      off = fma(t[5], x3m, off);
      const Ti ax = fma(t[6], x0, -off);
      if (MODE == ST_MATVEC) {
        out = ax;
        acc0.add_prod(x0, ax);
      } else {
        out = bv - ax;
        acc0.add_prod(out, out);
        acc1.add_prod(bv, bv);
      }
      xm = x0;
      x0 = xp;
    } else {
      out = bv;
      acc0.add_prod(bv, bv);
      acc1.add_prod(bv, bv);
    }
    y[base + row] = (To)out;
  }
}

}  // namespace sq
