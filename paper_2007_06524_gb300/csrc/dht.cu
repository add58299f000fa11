// Preconditioner apply z = F^-1 G F r (Sec. 4.2, Eq. 31) as five pencil passes.
//
// G(k1,k2,k3) depends on k only through lambda_k1 + lambda_k2 + lambda_k3 with
// lambda_k = lambda_{N-k}, so G is even in each index separately. Such a
// multiplier is also diagonal in the separable discrete Hartley basis
// cas(2 pi j k / N) = cos + sin, which is real and its own inverse up to N:
//   z = H3 (G .* H3 r) / N^3,  H3 = H (x) H (x) H.
// All passes therefore read and write real N^3 fields in the same layout, and
// r.z = sum_k G_k (H3 r)_k^2 / N^3 (Parseval) is reduced where the spectrum is
// in registers.
//
// A 1D Hartley transform of two real pencils a, b is taken from one complex
// FFT of a + i b (mixed-radix Stockham, radices 2/3/4/8, in shared memory):
//   2 (H a)_k = Re X_k - Im X_k + Re X_{N-k} + Im X_{N-k}
//   2 (H b)_k = Re X_k + Im X_k - Re X_{N-k} + Im X_{N-k}.
// The factor 2 per pass (2^6 over the six 1D transforms) and 1/N^3 are folded
// into G (scale = 1 / (64 N^3)).
//
// Passes (x3 is the contiguous axis):
//   A: x3 transform of r (PCG: r -= alpha q first, reducing ||r||^2)
//   B: x2 transform, in place
//   C: x1 transform, multiply by G on the fly (exact 1/(l1+l2+l3) or rank-R
//      sum_r u_r u_r u_r), reduce r.z, x1 transform again, in place
//   D: x2 transform, in place
//   E: x3 transform -> z (PCG: x += alpha p; p = z + beta p)
// A tile is P complex pencils = 2P real pencils: 2P adjacent rows for x3,
// 2P adjacent x3-columns for x1 and x2 (coalesced 2P-wide row segments).
#include "common.cuh"

namespace sq {

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C w) {
  return C{fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x)};
}
template <typename C>
__device__ __forceinline__ C mul_mi(C a) { return C{a.y, -a.x}; }  // (-i) a

template <typename T, typename C>
__device__ __forceinline__ void dft4(C &u0, C &u1, C &u2, C &u3) {
  const C t0 = cadd(u0, u2), t1 = csub(u0, u2), t2 = cadd(u1, u3), t3 = mul_mi(csub(u1, u3));
  u0 = cadd(t0, t2);
  u2 = csub(t0, t2);
  u1 = cadd(t1, t3);
  u3 = csub(t1, t3);
}

template <typename T, typename C, int R>
__device__ __forceinline__ void dft(C (&u)[R]) {
  if (R == 2) {
    const C t = u[0];
    u[0] = cadd(t, u[1]);
    u[1] = csub(t, u[1]);
  } else if (R == 3) {
    const T c = (T)0.86602540378443864676;  // sqrt(3)/2
    const C s = cadd(u[1], u[2]), d = csub(u[1], u[2]);
    const C m = C{fma((T)-0.5, s.x, u[0].x), fma((T)-0.5, s.y, u[0].y)};
    u[0] = cadd(u[0], s);
    u[1] = C{fma(c, d.y, m.x), fma(-c, d.x, m.y)};
    u[2] = C{fma(-c, d.y, m.x), fma(c, d.x, m.y)};
  } else if (R == 4) {
    dft4<T, C>(u[0], u[1], u[2], u[3]);
  } else if (R == 8) {
    const T h = (T)0.70710678118654752440;  // sqrt(2)/2
    C e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
    C o0 = u[1], o1 = u[3], o2 = u[5], o3 = u[7];
    dft4<T, C>(e0, e1, e2, e3);
    dft4<T, C>(o0, o1, o2, o3);
    const C w1 = C{h * (o1.x + o1.y), h * (o1.y - o1.x)};
    const C w2 = mul_mi(o2);
    const C w3 = C{h * (o3.y - o3.x), -h * (o3.x + o3.y)};
    u[0] = cadd(e0, o0);
    u[4] = csub(e0, o0);
    u[1] = cadd(e1, w1);
    u[5] = csub(e1, w1);
    u[2] = cadd(e2, w2);
    u[6] = csub(e2, w2);
    u[3] = cadd(e3, w3);
    u[7] = csub(e3, w3);
  }
}

// One radix-R Stockham stage over P pencils stored [j][p] with row stride SP.
// ps = product of the radices of the previous stages.
template <typename T, typename C, int R>
__device__ __forceinline__ void fft_stage(const C *__restrict__ in, C *__restrict__ out, const C *__restrict__ tw,
                                          int N, int ps, int SP, int logP) {
  const int P = 1 << logP;
  const int NR = N / R;
  const int nb = NR << logP;
  const int tstride = N / (ps * R);
  for (int t = threadIdx.x; t < nb; t += kThreads) {
    const int p = t & (P - 1);
    const int b = t >> logP;
    const int k = b % ps;
    C u[R];
#pragma unroll
    for (int q = 0; q < R; ++q) u[q] = in[(b + q * NR) * SP + p];
    if (ps > 1) {
      const int step = k * tstride;
#pragma unroll
      for (int q = 1; q < R; ++q) u[q] = cmul(u[q], tw[q * step]);
    }
    dft<T, C, R>(u);
    const int j = (b - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) out[(j + q * ps) * SP + p] = u[q];
  }
}

template <typename T, typename C>
__device__ __forceinline__ C *fft_all(C *b0, C *b1, const C *tw, const SpectralDev &sp, int SP, int logP) {
  C *src = b0, *dst = b1;
  int ps = 1;
  for (int s = 0; s < sp.nst; ++s) {
    const int r = sp.radix[s];
    switch (r) {
      case 2: fft_stage<T, C, 2>(src, dst, tw, sp.N, ps, SP, logP); break;
      case 3: fft_stage<T, C, 3>(src, dst, tw, sp.N, ps, SP, logP); break;
      case 4: fft_stage<T, C, 4>(src, dst, tw, sp.N, ps, SP, logP); break;
      default: fft_stage<T, C, 8>(src, dst, tw, sp.N, ps, SP, logP); break;
    }
    __syncthreads();
    C *t = src;
    src = dst;
    dst = t;
    ps *= r;
  }
  return src;
}

template <typename T>
struct DhtArgs {
  SpectralDev sp;
  const T *in;
  T *out;
  T *r;
  const T *q;
  T *p;
  T *x;
  RedBuf rb;
  int first;
  int check_done;
  int logP;
  int ntiles;
};

enum LoadMode { LD_PLAIN = 0, LD_RESID = 1 };
enum StoreMode { SO_PLAIN = 0, SO_PCG = 1 };

template <typename T, int AXIS, int LOADM, int STOREM, bool SCALE>
__global__ void __launch_bounds__(kThreads) k_dht(DhtArgs<T> a) {
  using C = typename Cx<T>::type;
  if (a.check_done && *(volatile int *)&a.rb.st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.sp.N;
  const int logP = a.logP;
  const int P = 1 << logP;
  const int SP = P + 1;
  C *buf0 = reinterpret_cast<C *>(smem_raw);
  C *buf1 = buf0 + N * SP;
  C *tw = buf1 + N * SP;
  T *vtab = reinterpret_cast<T *>(tw + N);  // rank x 2P column factors (pass C, rank-R)
  const int tid = threadIdx.x;
  const C *twg = reinterpret_cast<const C *>(a.sp.tw);
  for (int m = tid; m < N; m += kThreads) tw[m] = twg[m];

  const size_t NN = (size_t)N * N;
  const int nb2 = N / (2 * P);  // tiles per line for x1 / x2 passes
  const T alpha = (T)a.rb.st->alpha;
  const T beta = (T)a.rb.st->beta;
  const T *lam = reinterpret_cast<const T *>(a.sp.lam);
  const T *uf = reinterpret_cast<const T *>(a.sp.u);
  const int R = a.sp.rank;
  const T gscale = (T)a.sp.scale;
  double acc = 0.0;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    __syncthreads();
    // ------------------------------------------------------------------ load
    size_t base = 0, stride = 0;
    int k2 = 0, c0 = 0;
    if (AXIS == 3) {
      const size_t row0 = (size_t)tile * 2 * P;
      const int halfN = N >> 1;
      for (int e = tid; e < P * N; e += kThreads) {
        const int q = e / halfN;
        const int jj = 2 * (e - q * halfN);
        const size_t g = (row0 + q) * N + jj;
        using T2 = C;
        T2 v = reinterpret_cast<const T2 *>(a.in)[g >> 1];
        if (LOADM == LD_RESID && !a.first) {
          const T2 qq = reinterpret_cast<const T2 *>(a.q)[g >> 1];
          v.x = fma(-alpha, qq.x, v.x);
          v.y = fma(-alpha, qq.y, v.y);
          reinterpret_cast<T2 *>(a.r)[g >> 1] = v;
          acc = fma((double)v.x, (double)v.x, acc);
          acc = fma((double)v.y, (double)v.y, acc);
        }
        T *bs = reinterpret_cast<T *>(buf0);
        bs[(jj * SP + (q >> 1)) * 2 + (q & 1)] = v.x;
        bs[((jj + 1) * SP + (q >> 1)) * 2 + (q & 1)] = v.y;
      }
    } else {
      const int line = tile / nb2;
      const int cb = tile - line * nb2;
      c0 = cb * 2 * P;
      if (AXIS == 2) {
        base = (size_t)line * NN + c0;
        stride = N;
      } else {
        base = (size_t)line * N + c0;
        stride = NN;
        k2 = line;
      }
      for (int e = tid; e < P * N; e += kThreads) {
        const int p = e & (P - 1);
        const int j = e >> logP;
        const size_t g = base + (size_t)j * stride + 2 * p;
        buf0[j * SP + p] = reinterpret_cast<const C *>(a.in)[g >> 1];
      }
      if (SCALE && R > 0) {
        for (int e = tid; e < R * 2 * P; e += kThreads) {
          const int rr = e / (2 * P), w = e - rr * 2 * P;
          vtab[e] = uf[rr * N + k2] * uf[rr * N + c0 + w];
        }
      }
    }
    __syncthreads();
    // --------------------------------------------------------- transform(s)
    C *res = fft_all<T, C>(buf0, buf1, tw, a.sp, SP, logP);
    {
      const int halfN = N >> 1;
      for (int t = tid; t < ((halfN + 1) << logP); t += kThreads) {
        const int p = t & (P - 1);
        const int k = t >> logP;
        const int km = (k == 0) ? 0 : N - k;
        const C X = res[k * SP + p], Y = res[km * SP + p];
        T ak = X.x - X.y + Y.x + Y.y, bk = X.x + X.y - Y.x + Y.y;
        T akm = Y.x - Y.y + X.x + X.y, bkm = Y.x + Y.y - X.x + X.y;
        if (SCALE) {
          const int k3a = c0 + 2 * p, k3b = k3a + 1;
          T ga, gb;
          if (R == 0) {
            const T l12 = lam[k] + lam[k2];
            const T g1 = l12 + lam[k3a], g2 = l12 + lam[k3b];
            ga = (g1 > (T)0) ? gscale / g1 : (T)0;
            gb = (g2 > (T)0) ? gscale / g2 : (T)0;
          } else {
            T sa = (T)0, sb = (T)0;
            for (int rr = 0; rr < R; ++rr) {
              const T uk = uf[rr * N + k];
              sa = fma(uk, vtab[rr * 2 * P + 2 * p], sa);
              sb = fma(uk, vtab[rr * 2 * P + 2 * p + 1], sb);
            }
            ga = (k == 0 && k2 == 0 && k3a == 0) ? (T)0 : sa;
            gb = sb;  // k3b >= 1
          }
          double e2 = (double)ga * ((double)ak * ak) + (double)gb * ((double)bk * bk);
          if (km != k) e2 += (double)ga * ((double)akm * akm) + (double)gb * ((double)bkm * bkm);
          acc += e2;
          ak *= ga;
          akm *= ga;
          bk *= gb;
          bkm *= gb;
        }
        res[k * SP + p] = C{ak, bk};
        if (km != k) res[km * SP + p] = C{akm, bkm};
      }
      __syncthreads();
    }
    if (SCALE) {
      C *other = (res == buf0) ? buf1 : buf0;
      res = fft_all<T, C>(res, other, tw, a.sp, SP, logP);
      const int halfN = N >> 1;
      for (int t = tid; t < ((halfN + 1) << logP); t += kThreads) {
        const int p = t & (P - 1);
        const int k = t >> logP;
        const int km = (k == 0) ? 0 : N - k;
        const C X = res[k * SP + p], Y = res[km * SP + p];
        res[k * SP + p] = C{X.x - X.y + Y.x + Y.y, X.x + X.y - Y.x + Y.y};
        if (km != k) res[km * SP + p] = C{Y.x - Y.y + X.x + X.y, Y.x + Y.y - X.x + X.y};
      }
      __syncthreads();
    }
    // ----------------------------------------------------------------- store
    if (AXIS == 3) {
      const size_t row0 = (size_t)tile * 2 * P;
      const int halfN = N >> 1;
      const T *bs = reinterpret_cast<const T *>(res);
      for (int e = tid; e < P * N; e += kThreads) {
        const int q = e / halfN;
        const int jj = 2 * (e - q * halfN);
        const size_t g = (row0 + q) * N + jj;
        C z;
        z.x = bs[(jj * SP + (q >> 1)) * 2 + (q & 1)];
        z.y = bs[((jj + 1) * SP + (q >> 1)) * 2 + (q & 1)];
        if (STOREM == SO_PCG) {
          C *pp = reinterpret_cast<C *>(a.p) + (g >> 1);
          if (a.first) {
            *pp = z;
          } else {
            C *xx = reinterpret_cast<C *>(a.x) + (g >> 1);
            const C po = *pp;
            C xo = *xx;
            xo.x = fma(alpha, po.x, xo.x);
            xo.y = fma(alpha, po.y, xo.y);
            *xx = xo;
            *pp = C{fma(beta, po.x, z.x), fma(beta, po.y, z.y)};
          }
        } else {
          reinterpret_cast<C *>(a.out)[g >> 1] = z;
        }
      }
    } else {
      for (int e = tid; e < P * N; e += kThreads) {
        const int p = e & (P - 1);
        const int j = e >> logP;
        const size_t g = base + (size_t)j * stride + 2 * p;
        reinterpret_cast<C *>(a.out)[g >> 1] = res[j * SP + p];
      }
    }
  }

  if (LOADM == LD_RESID || SCALE) {
    double v[1] = {acc}, s[1];
    if (reduce_last_block<1>(v, a.rb.partials, &a.rb.st->ticket, s)) {
      if (tid == 0) {
        int op = FIN_NONE;
        if (LOADM == LD_RESID) op = a.first ? FIN_NONE : FIN_RR_ITER;
        if (SCALE) op = a.first ? FIN_RZ_FIRST : FIN_RZ_BETA;
        finalize_scalars(a.rb.st, op, s, 1);
      }
    }
  }
}

int dht_tile_pencils(int N, int elem_bytes) {
  // 2P real pencils per tile: 128-byte row segments where N allows, and two
  // ping-pong buffers of N (P+1) complex values within about 80 KB.
  int P = 128 / (2 * elem_bytes);
  while (P > 1 && ((N % (2 * P)) != 0 || 2L * N * (P + 1) * 2 * elem_bytes > 90 * 1024)) P >>= 1;
  return P;
}

static size_t dht_smem_bytes(int N, int P, int rank, int elem_bytes) {
  const size_t c = 2 * (size_t)elem_bytes;
  return 2 * (size_t)N * (P + 1) * c + (size_t)N * c + (size_t)rank * 2 * P * elem_bytes;
}

template <typename T, int AXIS, int LOADM, int STOREM, bool SCALE>
static cudaError_t launch_one(const DhtArgs<T> &a, int grid, size_t smem, cudaStream_t s) {
  auto kern = k_dht<T, AXIS, LOADM, STOREM, SCALE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dht_pass(int pass, const SpectralDev &sp, const T *in, T *out, T *r, const T *q, T *p, T *x,
                            RedBuf rb, bool first, bool check_done, cudaStream_t s) {
  const int N = sp.N;
  const int P = dht_tile_pencils(N, (int)sizeof(T));
  int logP = 0;
  while ((1 << logP) < P) ++logP;
  DhtArgs<T> a;
  a.sp = sp;
  a.in = in;
  a.out = out;
  a.r = r;
  a.q = q;
  a.p = p;
  a.x = x;
  a.rb = rb;
  a.first = first ? 1 : 0;
  a.check_done = check_done ? 1 : 0;
  a.logP = logP;
  a.ntiles = (int)(((long long)N * N) / (2 * P));
  const int grid = a.ntiles < 8192 ? a.ntiles : 8192;
  const size_t smem = dht_smem_bytes(N, P, pass == PASS_C ? sp.rank : 0, (int)sizeof(T));
  switch (pass) {
    case PASS_A_RESID: return launch_one<T, 3, LD_RESID, SO_PLAIN, false>(a, grid, smem, s);
    case PASS_A_PLAIN: return launch_one<T, 3, LD_PLAIN, SO_PLAIN, false>(a, grid, smem, s);
    case PASS_B: return launch_one<T, 2, LD_PLAIN, SO_PLAIN, false>(a, grid, smem, s);
    case PASS_C: return launch_one<T, 1, LD_PLAIN, SO_PLAIN, true>(a, grid, smem, s);
    case PASS_E_PCG: return launch_one<T, 3, LD_PLAIN, SO_PCG, false>(a, grid, smem, s);
    case PASS_E_PLAIN: return launch_one<T, 3, LD_PLAIN, SO_PLAIN, false>(a, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_dht_pass<double>(int, const SpectralDev &, const double *, double *, double *,
                                             const double *, double *, double *, RedBuf, bool, bool, cudaStream_t);
template cudaError_t launch_dht_pass<float>(int, const SpectralDev &, const float *, float *, float *, const float *,
                                            float *, float *, RedBuf, bool, bool, cudaStream_t);

}  // namespace sq
