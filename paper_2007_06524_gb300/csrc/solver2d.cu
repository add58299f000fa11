// The 2D corrector problem (the paper's 2D experiments, Sec. 5): the same
// method one dimension down, on an N x N periodic grid (x2 contiguous) with an
// L x L checkerboard of cells, N = L n up to 2048.
//
// Operator (Sec. 3 in 2D, lumped Q1): for node j,
//   (A x)(j) = sum_d a_d(j) (x(j) - x(j+e_d)) + a_d(j-e_d) (x(j) - x(j-e_d)),
// a_d(j) = mean of the two voxels beside the edge j -> j+e_d (voxel index j_d
// along d, j_t - 1 and j_t along the other axis). The four voxels around a
// node -- one bit each: bit s1*2 + s2 is voxel (j1-s1, j2-s2) -- fix its four
// edge coefficients and the diagonal through a 16-entry table. Sub-cell
// inclusions as in 3D: a voxel is high only if its cell is high and it lies in
// the cell's centred square [sub_lo, sub_hi)^2. RHS: b_i(j) = a_i(j) - a_i(j-e_i).
//
// Preconditioner (Sec. 4 in 2D): G(k1,k2) = 1/(l_k1 + l_k2), G(0,0) = 0, or
// the exponential sum sum_r w_r exp(-t_r (l_k1 + l_k2)), applied as a 2D
// Hartley transform in three passes: rows (fused r -= alpha q, ||r||^2),
// columns with the scaling in between (r.z), rows (fused x += alpha p,
// p = z + beta p). The passes are the 3D Hartley tiles of dht.cu with N rows;
// the column tile is the x2 tile of line 0, whose multiplier G(k, 0, k3) is
// G2(k, k3) once the factors and the scale 1/(16 N^2) (2^4 from the four 1D
// transforms, 1/N^2 from the inverse) are set for 2D.
//
// A_hom (Eq. 21 in 2D): A_ij = delta_ij mean(a_j) + mean(a_j D_j psi_i) and
// the energy form mean(sum_d a_d (delta_id + D_d psi_i)(delta_jd + D_d psi_j)).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace sq {
namespace {

constexpr int kMaxN2 = 2048;

bool valid_N2(int N) {
  if (N < 8 || N > kMaxN2 || (N & 1)) return false;
  int m = N;
  while (m % 2 == 0) m /= 2;
  if (m % 3 == 0) m /= 3;
  return m == 1;
}

struct Cells2D {
  const uint8_t *phase;  // L^2 cell phases, index c2 + L c1
  int L, n, N;
  int sub_lo, sub_hi;
  double edge[3];  // two voxels, k of them high: (k a_hi + (2-k) a_lo) / 2
  double diag[9];  // eight voxel slots of the four edges, K high: (K a_hi + (8-K) a_lo) / 2
};

// Table row m (4 voxel bits): 0 a_1(j), 1 a_1(j-e1), 2 a_2(j), 3 a_2(j-e2), 4 diagonal.
__device__ __forceinline__ void build_table_2d(double (*tab)[5], short *cell, uint8_t *ins, const Cells2D &c) {
  const unsigned face[4] = {0x3u, 0xCu, 0x5u, 0xAu};
  for (int m = threadIdx.x; m < 16; m += blockDim.x) {
    int kk = 0;
    for (int f = 0; f < 4; ++f) {
      const int k = __popc(m & face[f]);
      tab[m][f] = c.edge[k];
      kk += k;
    }
    tab[m][4] = c.diag[kk];
  }
  for (int v = threadIdx.x; v < c.N; v += blockDim.x) {
    const int cv = v / c.n, u = v - cv * c.n;
    cell[v] = (short)cv;
    ins[v] = (u >= c.sub_lo && u < c.sub_hi) ? 1 : 0;
  }
}

__device__ __forceinline__ unsigned node_bits(const Cells2D &c, const short *cell, const uint8_t *ins, int j1, int j1m,
                                              int j2, int j2m) {
  const uint8_t *r0 = c.phase + (size_t)cell[j1] * c.L, *r1 = c.phase + (size_t)cell[j1m] * c.L;
  const int ca = cell[j2], cb = cell[j2m];
  const bool a1 = ins[j1], b1 = ins[j1m], a2 = ins[j2], b2 = ins[j2m];
  return ((r0[ca] && a1 && a2) ? 1u : 0u) | ((r0[cb] && a1 && b2) ? 2u : 0u) | ((r1[ca] && b1 && a2) ? 4u : 0u) |
         ((r1[cb] && b1 && b2) ? 8u : 0u);
}

// One thread per column j2 over rows [z0, z1): y = A x (ST_MATVEC, reduces
// x.y), y = b_dir - A x (ST_RESID, reduces ||y||^2, ||b||^2), y = b_dir
// (ST_RHS, reduces ||b||^2 twice).
template <int MODE>
__global__ void __launch_bounds__(kThreads) k2_stencil(Cells2D c, int dir, const double *__restrict__ x,
                                                       double *__restrict__ y, RedBuf rb, int fin, int check_done,
                                                       int zc) {
  if (check_done && *(volatile int *)&rb.st->done) return;
  __shared__ double tab[16][5];
  __shared__ short cell[kMaxN2];
  __shared__ uint8_t ins[kMaxN2];
  build_table_2d(tab, cell, ins, c);
  __syncthreads();
  const int N = c.N;
  const int j2 = blockIdx.x * kThreads + threadIdx.x;
  const int z0 = blockIdx.y * zc, z1 = min(z0 + zc, N);
  double acc0 = 0.0, acc1 = 0.0;
  if (j2 < N) {
    const int j2m = (j2 == 0) ? N - 1 : j2 - 1, j2p = (j2 == N - 1) ? 0 : j2 + 1;
    const int j1m0 = (z0 == 0) ? N - 1 : z0 - 1;
    double xm = 0.0, x0 = 0.0;
    if (MODE != ST_RHS) {
      xm = x[(size_t)j1m0 * N + j2];
      x0 = x[(size_t)z0 * N + j2];
    }
    for (int j1 = z0; j1 < z1; ++j1) {
      const int j1m = (j1 == 0) ? N - 1 : j1 - 1, j1p = (j1 == N - 1) ? 0 : j1 + 1;
      const double *t = tab[node_bits(c, cell, ins, j1, j1m, j2, j2m)];
      const size_t o = (size_t)j1 * N;
      const double bv = (dir == 0) ? t[0] - t[1] : t[2] - t[3];
      double out;
      if (MODE != ST_RHS) {
        const double xp = x[(size_t)j1p * N + j2];
        const double xe = x[o + j2p], xw = x[o + j2m];
        double off = t[0] * xp;
        off = fma(t[1], xm, off);
        off = fma(t[2], xe, off);
        off = fma(t[3], xw, off);
        const double ax = fma(t[4], x0, -off);
        if (MODE == ST_MATVEC) {
          out = ax;
          acc0 = fma(x0, ax, acc0);
        } else {
          out = bv - ax;
          acc0 = fma(out, out, acc0);
          acc1 = fma(bv, bv, acc1);
        }
        xm = x0;
        x0 = xp;
      } else {
        out = bv;
        acc0 = fma(bv, bv, acc0);
        acc1 = fma(bv, bv, acc1);
      }
      y[o + j2] = out;
    }
  }
  double v[2] = {acc0, acc1}, s[2];
  if (reduce_last_block<2>(v, rb.partials, &rb.st->ticket, s)) {
    if (threadIdx.x == 0) finalize_scalars(rb.st, fin, s, 2);
  }
}

// Reduced quantities: 0..3 M[i][d] = sum a_d D_d psi_i, 4..5 sum a_d, 6..8
// energy sums for (i,j) in (00, 01, 11).
__global__ void __launch_bounds__(kThreads) k2_ahom(Cells2D c, const double *__restrict__ p0,
                                                    const double *__restrict__ p1, RedBuf rb, int zc) {
  __shared__ double tab[16][5];
  __shared__ short cell[kMaxN2];
  __shared__ uint8_t ins[kMaxN2];
  build_table_2d(tab, cell, ins, c);
  __syncthreads();
  const int N = c.N;
  const int j2 = blockIdx.x * kThreads + threadIdx.x;
  const int z0 = blockIdx.y * zc, z1 = min(z0 + zc, N);
  double acc[9];
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  if (j2 < N) {
    const int j2m = (j2 == 0) ? N - 1 : j2 - 1, j2p = (j2 == N - 1) ? 0 : j2 + 1;
    const double *ps[2] = {p0, p1};
    for (int j1 = z0; j1 < z1; ++j1) {
      const int j1m = (j1 == 0) ? N - 1 : j1 - 1, j1p = (j1 == N - 1) ? 0 : j1 + 1;
      const double *t = tab[node_bits(c, cell, ins, j1, j1m, j2, j2m)];
      const double a[2] = {t[0], t[2]};
      const size_t o = (size_t)j1 * N + j2, on[2] = {(size_t)j1p * N + j2, (size_t)j1 * N + j2p};
      double g[2][2];
      for (int i = 0; i < 2; ++i)
        for (int d = 0; d < 2; ++d) g[i][d] = ps[i][on[d]] - ps[i][o];
      for (int i = 0; i < 2; ++i)
        for (int d = 0; d < 2; ++d) acc[2 * i + d] = fma(a[d], g[i][d], acc[2 * i + d]);
      acc[4] += a[0];
      acc[5] += a[1];
      int q = 6;
      for (int i = 0; i < 2; ++i)
        for (int jj = i; jj < 2; ++jj) {
          double e = 0.0;
          for (int d = 0; d < 2; ++d)
            e += a[d] * ((i == d ? 1.0 : 0.0) + g[i][d]) * ((jj == d ? 1.0 : 0.0) + g[jj][d]);
          acc[q++] += e;
        }
    }
  }
  double s[9];
  if (reduce_last_block<9>(acc, rb.partials, &rb.st->ticket, s)) {
    if (threadIdx.x == 0) finalize_scalars(rb.st, FIN_NONE, s, 9);
  }
}

__global__ void k2_scalars_reset(Scalars *st, double tolrel2, int max_iter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    Scalars z;
    memset(&z, 0, sizeof(z));
    z.tolrel2 = tolrel2;
    z.max_iter = max_iter;
    *st = z;
  }
}

// Row chunk of the stencil and A_hom sweeps: about 2 K blocks.
int rows_per_block(int N) {
  const int nbx = (N + kThreads - 1) / kThreads;
  int zc = (N * nbx + 2047) / 2048;
  if (zc < 1) zc = 1;
  if (zc > N) zc = N;
  return zc;
}

}  // namespace
}  // namespace sq

using namespace sq;

struct sq2d_coeffs {
  int L, n, N;
  double a_lo, a_hi;
  int sub_lo = 0, sub_hi = 1 << 30;
  uint8_t *d_phase = nullptr;
  cudaStream_t stream = nullptr;
  Scalars *d_st = nullptr;
  double *d_partials = nullptr;
  Scalars *h_st = nullptr;
};

struct sq2d_precond {
  int N, rank;
  std::vector<double> t, w;
  SpectralDev sp;
  void *d_mem = nullptr;
};

struct sq2d_workspace {
  int N;
  double *f = nullptr;  // r, p, q, Y
  Scalars *d_st = nullptr;
  double *d_partials = nullptr;
  Scalars *h_st = nullptr;
  int *h_poll = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // CUDA graphs of kPollChunk iterations (see loop2d) with their signatures
  struct IterGraph {
    std::vector<uint64_t> sig;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
  };
  std::vector<IterGraph> graphs;
};

namespace {

Cells2D cells2d(const sq2d_coeffs *c) {
  Cells2D d;
  d.phase = c->d_phase;
  d.L = c->L;
  d.n = c->n;
  d.N = c->N;
  d.sub_lo = c->sub_lo;
  d.sub_hi = c->sub_hi;
  for (int k = 0; k <= 2; ++k) d.edge[k] = (k * c->a_hi + (2 - k) * c->a_lo) * 0.5;
  for (int k = 0; k <= 8; ++k) d.diag[k] = (k * c->a_hi + (8 - k) * c->a_lo) * 0.5;
  return d;
}

RedBuf rbuf(Scalars *st, double *partials) {
  RedBuf rb;
  rb.st = st;
  rb.partials = partials;
  return rb;
}

cudaError_t launch_stencil2d(const Cells2D &c, int mode, int dir, const double *x, double *y, RedBuf rb, int fin,
                             bool check_done, cudaStream_t s) {
  const int N = c.N, zc = rows_per_block(N);
  const dim3 grid((N + kThreads - 1) / kThreads, (N + zc - 1) / zc);
  const int cd = check_done ? 1 : 0;
  switch (mode) {
    case ST_MATVEC: k2_stencil<ST_MATVEC><<<grid, kThreads, 0, s>>>(c, dir, x, y, rb, fin, cd, zc); break;
    case ST_RESID: k2_stencil<ST_RESID><<<grid, kThreads, 0, s>>>(c, dir, x, y, rb, fin, cd, zc); break;
    default: k2_stencil<ST_RHS><<<grid, kThreads, 0, s>>>(c, dir, x, y, rb, fin, cd, zc); break;
  }
  return cudaGetLastError();
}

#define SQ2_CK(call)                           \
  do {                                         \
    if ((call) != cudaSuccess) return SQ_ECUDA; \
  } while (0)

int read2(Scalars *h, const Scalars *d, cudaStream_t s) {
  SQ2_CK(cudaMemcpyAsync(h, d, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  SQ2_CK(cudaStreamSynchronize(s));
  return SQ_OK;
}

int precond_first2d(const sq2d_precond *pc, double *r, double *Y, double *p, RedBuf rb, cudaStream_t s) {
  SQ2_CK(launch_dht_pass_2d<double>(PASS_A_PLAIN, pc->sp, r, Y, nullptr, nullptr, nullptr, nullptr, rb, true, true, s));
  SQ2_CK(launch_dht_pass_2d<double>(PASS_C, pc->sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, true, true, s));
  SQ2_CK(launch_dht_pass_2d<double>(PASS_E_PCG, pc->sp, Y, nullptr, nullptr, nullptr, p, nullptr, rb, true, true, s));
  return SQ_OK;
}

int iteration2d(const Cells2D &cd, const sq2d_precond *pc, double *x, double *r, double *p, double *q, double *Y,
                RedBuf rb, cudaStream_t s) {
  SQ2_CK(launch_stencil2d(cd, ST_MATVEC, 0, p, q, rb, FIN_ALPHA, true, s));
  SQ2_CK(launch_dht_pass_2d<double>(PASS_A_RESID, pc->sp, r, Y, r, q, nullptr, nullptr, rb, false, true, s));
  SQ2_CK(launch_dht_pass_2d<double>(PASS_C, pc->sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, false, true, s));
  SQ2_CK(launch_dht_pass_2d<double>(PASS_E_PCG, pc->sp, Y, nullptr, nullptr, nullptr, p, x, rb, false, true, s));
  return SQ_OK;
}

// A chunk of iterations as one replayed CUDA graph, as for the 3D solves
// (SQ_OPT_PCG_GRAPHS): found by a signature of every launch parameter it
// bakes in (fields, reduction buffers, the cell and spectral descriptors,
// the option epoch), or captured on a private stream.
int graph2d(sq2d_workspace *w, const Cells2D &cd, const sq2d_precond *pc, double *x, double *r, double *p, double *q,
            double *Y, RedBuf rb, cudaGraphExec_t *exec) {
  std::vector<uint64_t> sig;
  auto add = [&](uint64_t u) { sig.push_back(u); };
  auto addp = [&](const void *ptr) { add((uint64_t)(uintptr_t)ptr); };
  auto addd = [&](double d) {
    uint64_t u;
    memcpy(&u, &d, sizeof(u));
    add(u);
  };
  add((uint64_t)option_epoch());
  addp(x), addp(r), addp(p), addp(q), addp(Y), addp(rb.st), addp(rb.partials);
  addp(cd.phase), add(cd.L), add(cd.n), add(cd.N), add((uint64_t)cd.sub_lo), add((uint64_t)cd.sub_hi);
  for (double e : cd.edge) addd(e);
  for (double e : cd.diag) addd(e);
  add(pc->sp.N), add(pc->sp.rank), addp(pc->sp.tw), addp(pc->sp.lam), addp(pc->sp.u), addd(pc->sp.scale);
  addp(pc->sp.gtab);
  for (const sq2d_workspace::IterGraph &e : w->graphs) {
    if (e.sig == sig) {
      *exec = e.exec;
      return SQ_OK;
    }
  }
  if (w->graphs.size() >= 8) {
    cudaGraphExecDestroy(w->graphs.front().exec);
    cudaGraphDestroy(w->graphs.front().graph);
    w->graphs.erase(w->graphs.begin());
  }
  cudaStream_t cs;
  SQ2_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int st = SQ_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = SQ_ECUDA;
  for (int i = 0; st == SQ_OK && i < kPollChunk; ++i) st = iteration2d(cd, pc, x, r, p, q, Y, rb, cs);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g) st = SQ_ECUDA;
  cudaGraphExec_t ge = nullptr;
  if (st == SQ_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) st = SQ_ECUDA;
  cudaStreamDestroy(cs);
  if (st != SQ_OK) {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    return st;
  }
  w->graphs.push_back(sq2d_workspace::IterGraph{std::move(sig), g, ge});
  *exec = ge;
  return SQ_OK;
}

// Iterations in chunks of kPollChunk, polling the device's stop flag one chunk behind.
int loop2d(sq2d_workspace *w, const Cells2D &cd, const sq2d_precond *pc, double *x, double *r, double *p, double *q,
           double *Y, RedBuf rb, int budget, cudaStream_t s) {
  const int chunk = kPollChunk;
  int launched = 0, slot = 0;
  bool pending[2] = {false, false};
  w->h_poll[0] = w->h_poll[1] = 0;
  const size_t done_off = offsetof(Scalars, done);
  cudaGraphExec_t gx = nullptr;
  if (pcg_graphs_enabled() && budget >= chunk) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SQ2_CK(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone && graph2d(w, cd, pc, x, r, p, q, Y, rb, &gx) != SQ_OK) {
      gx = nullptr;  // no graph (capture or instantiation failed): launch one by one
      (void)cudaGetLastError();
    }
  }
  while (launched < budget) {
    const int nb = (budget - launched < chunk) ? budget - launched : chunk;
    if (gx && nb == chunk) {
      SQ2_CK(cudaGraphLaunch(gx, s));
    } else {
      for (int i = 0; i < nb; ++i) {
        const int st = iteration2d(cd, pc, x, r, p, q, Y, rb, s);
        if (st != SQ_OK) return st;
      }
    }
    launched += nb;
    SQ2_CK(cudaMemcpyAsync(&w->h_poll[slot], reinterpret_cast<char *>(rb.st) + done_off, sizeof(int),
                           cudaMemcpyDeviceToHost, s));
    SQ2_CK(cudaEventRecord(w->ev[slot], s));
    pending[slot] = true;
    const int other = slot ^ 1;
    if (pending[other]) {
      SQ2_CK(cudaEventSynchronize(w->ev[other]));
      pending[other] = false;
      if (w->h_poll[other]) break;
    }
    slot = other;
  }
  return SQ_OK;
}

int alloc_coeffs2d(int L, int n, double a_lo, double a_hi, cudaStream_t s, sq2d_coeffs **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (L < 1 || n < 2 || !valid_N2(L * n)) return SQ_EINVAL;
  if (!(a_lo > 0.0) || !(a_hi > 0.0) || !std::isfinite(a_lo) || !std::isfinite(a_hi)) return SQ_EINVAL;
  sq2d_coeffs *c = new (std::nothrow) sq2d_coeffs();
  if (!c) return SQ_ENOMEM;
  c->L = L;
  c->n = n;
  c->N = L * n;
  c->a_lo = a_lo;
  c->a_hi = a_hi;
  c->stream = s;
  if (cudaMalloc(&c->d_phase, (size_t)L * L) != cudaSuccess || cudaMalloc(&c->d_st, sizeof(Scalars)) != cudaSuccess ||
      cudaMalloc(&c->d_partials, sizeof(double) * kMaxQ * kMaxPartials) != cudaSuccess ||
      cudaMallocHost(&c->h_st, sizeof(Scalars)) != cudaSuccess || cudaMemsetAsync(c->d_st, 0, sizeof(Scalars), s) != cudaSuccess) {
    sq2d_coeffs_destroy(c);
    return SQ_ENOMEM;
  }
  *out = c;
  return SQ_OK;
}

}  // namespace

extern "C" {

int sq2d_build_coeffs(int L, int n, uint64_t seed, double p_hi, double a_lo, double a_hi, sq_stream_t stream,
                      sq2d_coeffs **out) {
  if (!(p_hi >= 0.0 && p_hi <= 1.0)) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = alloc_coeffs2d(L, n, a_lo, a_hi, s, out);
  if (st != SQ_OK) return st;
  const uint64_t thr[3] = {(uint64_t)(p_hi * 9007199254740992.0), 0, 0};  // floor(p_hi * 2^53)
  if (launch_coeff_gen_cells((*out)->d_phase, L * L, seed, thr, s) != cudaSuccess) {
    sq2d_coeffs_destroy(*out);
    *out = nullptr;
    return SQ_ECUDA;
  }
  return SQ_OK;
}

int sq2d_coeffs_from_host(int L, int n, const uint8_t *host_phase, double a_lo, double a_hi, sq_stream_t stream,
                          sq2d_coeffs **out) {
  if (!host_phase) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = alloc_coeffs2d(L, n, a_lo, a_hi, s, out);
  if (st != SQ_OK) return st;
  std::vector<uint8_t> norm((size_t)L * L);
  for (size_t i = 0; i < norm.size(); ++i) norm[i] = host_phase[i] ? 1 : 0;
  if (cudaMemcpyAsync((*out)->d_phase, norm.data(), norm.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    sq2d_coeffs_destroy(*out);
    *out = nullptr;
    return SQ_ECUDA;
  }
  return SQ_OK;
}

int sq2d_coeffs_set_subcell(sq2d_coeffs *c, int sub) {
  if (!c || sub < 1 || sub > c->n || (c->n - sub) % 2 != 0) return SQ_EINVAL;
  if (sub == c->n) {
    c->sub_lo = 0;
    c->sub_hi = 1 << 30;
  } else {
    c->sub_lo = (c->n - sub) / 2;
    c->sub_hi = c->sub_lo + sub;
  }
  return SQ_OK;
}

int sq2d_coeffs_cells(const sq2d_coeffs *c, uint8_t *host_phase) {
  if (!c || !host_phase) return SQ_EINVAL;
  SQ2_CK(cudaMemcpyAsync(host_phase, c->d_phase, (size_t)c->L * c->L, cudaMemcpyDeviceToHost, c->stream));
  SQ2_CK(cudaStreamSynchronize(c->stream));
  return SQ_OK;
}

void sq2d_coeffs_destroy(sq2d_coeffs *c) {
  if (!c) return;
  if (c->d_phase) cudaFree(c->d_phase);
  if (c->d_st) cudaFree(c->d_st);
  if (c->d_partials) cudaFree(c->d_partials);
  if (c->h_st) cudaFreeHost(c->h_st);
  delete c;
}

int sq2d_precond_setup(int N, int rank, sq2d_precond **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (!valid_N2(N) || rank < 0 || rank == 1 || rank > kMaxExpRank) return SQ_EINVAL;
  const double pi = 3.14159265358979323846;
  const int R = rank;
  std::vector<double> tw(2 * N), lam(N), u((size_t)3 * (R > 0 ? R : 1) * N, 0.0), t, w;
  for (int m = 0; m < N; ++m) {
    tw[2 * m] = std::cos(2.0 * pi * m / N);
    tw[2 * m + 1] = -std::sin(2.0 * pi * m / N);
    const double sn = std::sin(pi * m / N);
    lam[m] = 4.0 * sn * sn;
  }
  if (R > 0) {
    exp_sum_nodes(N, R, 2, t, w);
    // x1 and x2 factors carry w^(1/3) exp(-t l) / (4 N) each; the middle factor
    // is read at index 0 only and carries w^(1/3): the product is
    // w exp(-t (l_k1 + l_k2)) / (16 N^2)
    for (int r = 0; r < R; ++r) {
      const double c3 = std::cbrt(w[r]);
      for (int k = 0; k < N; ++k) {
        const double e = c3 * std::exp(-t[r] * lam[k]);
        u[(size_t)r * N + k] = e / (4.0 * N);
        u[((size_t)R + r) * N + k] = e;
        u[((size_t)2 * R + r) * N + k] = e / (4.0 * N);
      }
    }
  }
  sq2d_precond *pc = new (std::nothrow) sq2d_precond();
  if (!pc) return SQ_ENOMEM;
  pc->N = N;
  pc->rank = R;
  pc->t = t;
  pc->w = w;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_tw = tw.size() * 8, b_lam = lam.size() * 8, b_u = u.size() * 8;
  if (cudaMalloc(&pc->d_mem, al(b_tw) + al(b_lam) + al(b_u)) != cudaSuccess) {
    delete pc;
    return SQ_ENOMEM;
  }
  char *bp = static_cast<char *>(pc->d_mem);
  if (cudaMemcpy(bp, tw.data(), b_tw, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(bp + al(b_tw), lam.data(), b_lam, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(bp + al(b_tw) + al(b_lam), u.data(), b_u, cudaMemcpyHostToDevice) != cudaSuccess) {
    sq2d_precond_destroy(pc);
    return SQ_ECUDA;
  }
  std::memset(&pc->sp, 0, sizeof(pc->sp));
  pc->sp.N = N;
  pc->sp.rank = R;
  pc->sp.nst = radix_plan_of(N, pc->sp.radix);
  pc->sp.scale = 1.0 / (16.0 * (double)N * N);
  pc->sp.tw = bp;
  pc->sp.lam = bp + al(b_tw);
  pc->sp.u = bp + al(b_tw) + al(b_lam);
  *out = pc;
  return SQ_OK;
}

int sq2d_precond_factors(const sq2d_precond *p, double *t, double *w) {
  if (!p) return SQ_EINVAL;
  for (int r = 0; r < p->rank; ++r) {
    if (t) t[r] = p->t[r];
    if (w) w[r] = p->w[r];
  }
  return SQ_OK;
}

void sq2d_precond_destroy(sq2d_precond *p) {
  if (!p) return;
  if (p->d_mem) cudaFree(p->d_mem);
  delete p;
}

int sq2d_workspace_create(int N, sq2d_workspace **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (!valid_N2(N)) return SQ_EINVAL;
  sq2d_workspace *w = new (std::nothrow) sq2d_workspace();
  if (!w) return SQ_ENOMEM;
  w->N = N;
  const size_t n2 = (size_t)N * N;
  if (cudaMalloc(&w->f, 4 * n2 * sizeof(double)) != cudaSuccess || cudaMalloc(&w->d_st, sizeof(Scalars)) != cudaSuccess ||
      cudaMalloc(&w->d_partials, sizeof(double) * kMaxQ * kMaxPartials) != cudaSuccess ||
      cudaMallocHost(&w->h_st, sizeof(Scalars)) != cudaSuccess || cudaMallocHost(&w->h_poll, 2 * sizeof(int)) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    sq2d_workspace_destroy(w);
    return SQ_ENOMEM;
  }
  *out = w;
  return SQ_OK;
}

void sq2d_workspace_destroy(sq2d_workspace *w) {
  if (!w) return;
  if (w->f) cudaFree(w->f);
  if (w->d_st) cudaFree(w->d_st);
  if (w->d_partials) cudaFree(w->d_partials);
  if (w->h_st) cudaFreeHost(w->h_st);
  if (w->h_poll) cudaFreeHost(w->h_poll);
  for (int i = 0; i < 2; ++i)
    if (w->ev[i]) cudaEventDestroy(w->ev[i]);
  for (sq2d_workspace::IterGraph &e : w->graphs) {
    cudaGraphExecDestroy(e.exec);
    cudaGraphDestroy(e.graph);
  }
  delete w;
}

int sq2d_pcg_solve(const sq2d_coeffs *c, const sq2d_precond *pc, sq2d_workspace *w, int dir, double tol, int max_iter,
                   double *psi, sq_solve_info *info, sq_stream_t stream) {
  if (!c || !pc || !w || !psi || (dir != 0 && dir != 1) || !(tol > 0.0) || max_iter < 1) return SQ_EINVAL;
  if (c->N != pc->N || c->N != w->N) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long n2 = (long long)c->N * c->N;
  double *r = w->f, *p = r + n2, *q = p + n2, *Y = q + n2;
  const RedBuf rb = rbuf(w->d_st, w->d_partials);
  const Cells2D cd = cells2d(c);
  k2_scalars_reset<<<1, 1, 0, s>>>(rb.st, tol * tol, max_iter);
  SQ2_CK(cudaGetLastError());
  SQ2_CK(cudaMemsetAsync(psi, 0, sizeof(double) * n2, s));
  SQ2_CK(launch_stencil2d(cd, ST_RHS, dir, nullptr, r, rb, FIN_RESID, false, s));
  Scalars *h = w->h_st;
  for (int restart = 0; restart < 4; ++restart) {
    int st = precond_first2d(pc, r, Y, p, rb, s);
    if (st != SQ_OK) return st;
    st = loop2d(w, cd, pc, psi, r, p, q, Y, rb, max_iter, s);
    if (st != SQ_OK) return st;
    SQ2_CK(launch_x_final_sum<double>(psi, p, rb, n2, s));
    SQ2_CK(launch_sub_mean<double>(psi, rb, n2, s));
    SQ2_CK(launch_stencil2d(cd, ST_RESID, dir, psi, r, rb, FIN_RESID, false, s));
    st = read2(h, rb.st, s);
    if (st != SQ_OK) return st;
    if (h->done || h->iter >= max_iter || h->breakdown) break;
  }
  const double relres_true = (h->bb > 0.0) ? std::sqrt(h->rr_true / h->bb) : 0.0;
  if (info) {
    info->iters = h->iter;
    info->outer_steps = 1;
    info->used_guess = 0;
    info->relres = (h->bb > 0.0) ? std::sqrt(h->rr / h->bb) : 0.0;
    info->relres_true = relres_true;
    info->status = (h->bb == 0.0 || relres_true <= tol) ? SQ_OK : SQ_ENOCONV;
  }
  return (h->bb == 0.0 || relres_true <= tol) ? SQ_OK : SQ_ENOCONV;
}

int sq2d_homogenized_matrix(const sq2d_coeffs *c, const double *psi0, const double *psi1, double *A_hom,
                            double *A_energy) {
  if (!c || !psi0 || !psi1 || !A_hom) return SQ_EINVAL;
  cudaStream_t s = c->stream;
  const Cells2D cd = cells2d(c);
  const int N = c->N, zc = rows_per_block(N);
  const dim3 grid((N + kThreads - 1) / kThreads, (N + zc - 1) / zc);
  k2_ahom<<<grid, kThreads, 0, s>>>(cd, psi0, psi1, rbuf(c->d_st, c->d_partials), zc);
  SQ2_CK(cudaGetLastError());
  const int st = read2(c->h_st, c->d_st, s);
  if (st != SQ_OK) return st;
  const double *red = c->h_st->red;
  const double inv = 1.0 / ((double)N * N);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) A_hom[2 * i + j] = ((i == j) ? red[4 + j] : 0.0) * inv + red[2 * i + j] * inv;
  if (A_energy) {
    A_energy[0] = red[6] * inv;
    A_energy[1] = A_energy[2] = red[7] * inv;
    A_energy[3] = red[8] * inv;
  }
  return SQ_OK;
}

int sq2d_apply_operator(const sq2d_coeffs *c, const double *x, double *y, sq_stream_t stream) {
  if (!c || !x || !y) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SQ2_CK(launch_stencil2d(cells2d(c), ST_MATVEC, 0, x, y, rbuf(c->d_st, c->d_partials), FIN_NONE, false, s));
  return SQ_OK;
}

int sq2d_rhs(const sq2d_coeffs *c, int dir, double *b, sq_stream_t stream) {
  if (!c || !b || (dir != 0 && dir != 1)) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SQ2_CK(launch_stencil2d(cells2d(c), ST_RHS, dir, nullptr, b, rbuf(c->d_st, c->d_partials), FIN_NONE, false, s));
  return SQ_OK;
}

int sq2d_apply_precond(const sq2d_precond *pc, sq2d_workspace *w, const double *r, double *z, sq_stream_t stream) {
  if (!pc || !w || !r || !z || pc->N != w->N) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const RedBuf rb = rbuf(w->d_st, w->d_partials);
  k2_scalars_reset<<<1, 1, 0, s>>>(rb.st, 0.0, 1);
  SQ2_CK(cudaGetLastError());
  double *Y = w->f + 3 * (size_t)pc->N * pc->N;
  SQ2_CK(launch_dht_pass_2d<double>(PASS_A_PLAIN, pc->sp, r, Y, nullptr, nullptr, nullptr, nullptr, rb, true, false, s));
  SQ2_CK(launch_dht_pass_2d<double>(PASS_C, pc->sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, true, false, s));
  SQ2_CK(launch_dht_pass_2d<double>(PASS_E_PLAIN, pc->sp, Y, z, nullptr, nullptr, nullptr, nullptr, rb, true, false, s));
  return SQ_OK;
}

}  // extern "C"
