// Device core of the Hartley-transform pencil passes, shared by the
// single-solve and the batched kernels. See dht.cu for the method.
#pragma once

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

// FP32 complex sums and differences as one packed two-lane instruction
// (add / sub .f32x2, sm_100 and later): fewer issued instructions in every
// butterfly of the FP32 passes. A complex product would need both operands
// broadcast into lane pairs first, so it stays scalar.
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
template <>
__device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}
template <>
__device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}

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
  } else if (R == 16) {
    // 16 = 4 x 4: DFT4 over the stride-4 subsequences, twiddles W16^(n2 k1),
    // DFT4 across them; output k1 + 4 k2.
    const T c = (T)0.92387953251128675613, s = (T)0.38268343236508977173, h = (T)0.70710678118654752440;
    C y[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C a0 = u[n2], a1 = u[4 + n2], a2 = u[8 + n2], a3 = u[12 + n2];
      dft4<T, C>(a0, a1, a2, a3);
      y[n2 * 4 + 0] = a0;
      y[n2 * 4 + 1] = a1;
      y[n2 * 4 + 2] = a2;
      y[n2 * 4 + 3] = a3;
    }
    y[5] = cmul(y[5], C{c, -s});    // W^1
    y[6] = cmul(y[6], C{h, -h});    // W^2
    y[7] = cmul(y[7], C{s, -c});    // W^3
    y[9] = cmul(y[9], C{h, -h});    // W^2
    y[10] = mul_mi(y[10]);          // W^4
    y[11] = cmul(y[11], C{-h, -h}); // W^6
    y[13] = cmul(y[13], C{s, -c});  // W^3
    y[14] = cmul(y[14], C{-h, -h}); // W^6
    y[15] = cmul(y[15], C{-c, s});  // W^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C b0 = y[k1], b1 = y[4 + k1], b2 = y[8 + k1], b3 = y[12 + k1];
      dft4<T, C>(b0, b1, b2, b3);
      u[k1] = b0;
      u[k1 + 4] = b1;
      u[k1 + 8] = b2;
      u[k1 + 12] = b3;
    }
  } else if (R == 6) {
    // 6 = 2 x 3: DFT3 of the even and odd samples, twiddles W6^k, radix-2 combine
    const T h = (T)0.5, c = (T)0.86602540378443864676;  // cos, sin of pi/3
    C e[3] = {u[0], u[2], u[4]}, o[3] = {u[1], u[3], u[5]};
    dft<T, C, 3>(e);
    dft<T, C, 3>(o);
    const C w1 = cmul(o[1], C{h, -c}), w2 = cmul(o[2], C{-h, -c});
    u[0] = cadd(e[0], o[0]);
    u[3] = csub(e[0], o[0]);
    u[1] = cadd(e[1], w1);
    u[4] = csub(e[1], w1);
    u[2] = cadd(e[2], w2);
    u[5] = csub(e[2], w2);
  } else if (R == 32) {
    // 32 = 4 x 8: DFT8 over the stride-4 subsequences, twiddles W32^(n2 k1),
    // DFT4 across them; output k1 + 8 k2. W32^j = (cos, -sin)(2 pi j / 32).
    const T c1 = (T)0.98078528040323044913, s1 = (T)0.19509032201612826785;
    const T c2 = (T)0.92387953251128675613, s2 = (T)0.38268343236508977173;
    const T c3 = (T)0.83146961230254523708, s3 = (T)0.55557023301960222474;
    const T h = (T)0.70710678118654752440;
    // cos and sin of 2 pi j / 32 for j = 0..21 (the twiddle exponents n2 k1 < 22)
    const T cs[22] = {(T)1, c1, c2, c3, h, s3, s2, s1, (T)0, -s1, -s2, -s3, -h, -c3, -c2, -c1, (T)-1, -c1, -c2, -c3, -h, -s3};
    const T sn[22] = {(T)0, s1, s2, s3, h, c3, c2, c1, (T)1, c1, c2, c3, h, s3, s2, s1, (T)0, -s1, -s2, -s3, -h, -c3};
    C y[4][8];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      C a[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) a[m] = u[n2 + 4 * m];
      dft<T, C, 8>(a);
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) {
        const int j = n2 * k1;
        y[n2][k1] = (j == 0) ? a[k1] : cmul(a[k1], C{cs[j], -sn[j]});
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
      C b0 = y[0][k1], b1 = y[1][k1], b2 = y[2][k1], b3 = y[3][k1];
      dft4<T, C>(b0, b1, b2, b3);
      u[k1] = b0;
      u[k1 + 8] = b1;
      u[k1 + 16] = b2;
      u[k1 + 24] = b3;
    }
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

// Twiddled butterflies with the complex products fused into the first layer
// of sums (FP64 stages): a + w b costs four FMAs (a complex product and a sum
// would cost six), and its partner a - w b = 2a - (a + w b) two more.
template <typename C>
__device__ __forceinline__ C cfma(C w, C b, C a) {
  return C{fma(w.x, b.x, fma(-w.y, b.y, a.x)), fma(w.x, b.y, fma(w.y, b.x, a.y))};
}
template <typename T, typename C>
__device__ __forceinline__ C ctwice_minus(C a, C s) {
  return C{fma((T)2, a.x, -s.x), fma((T)2, a.y, -s.y)};
}
// The 4-point DFT of (u0, w1 u1, w2 u2, w3 u3), in place (dft4's order).
template <typename T, typename C>
__device__ __forceinline__ void dft4_tw(C &u0, C &u1, C &u2, C &u3, C w1, C w2, C w3) {
  const C t0 = cfma(w2, u2, u0);                        // u0 + w2 u2
  const C t1 = ctwice_minus<T>(u0, t0);                 // u0 - w2 u2
  const C c = cmul(u1, w1);
  const C t2 = cfma(w3, u3, c);                         // w1 u1 + w3 u3
  const C t3 = mul_mi(ctwice_minus<T>(c, t2));          // -i (w1 u1 - w3 u3)
  u0 = cadd(t0, t2);
  u2 = csub(t0, t2);
  u1 = cadd(t1, t3);
  u3 = csub(t1, t3);
}
// dft<R> of (u0, w[1] u1, .., w[R-1] u_{R-1}) for R = 2, 4, 8 (dft's output order).
template <typename T, typename C, int R>
__device__ __forceinline__ void dft_tw(C (&u)[R], const C (&w)[R]) {
  if constexpr (R == 2) {
    const C s = cfma(w[1], u[1], u[0]);
    u[1] = ctwice_minus<T>(u[0], s);
    u[0] = s;
  } else if constexpr (R == 4) {
    dft4_tw<T, C>(u[0], u[1], u[2], u[3], w[1], w[2], w[3]);
  } else {
    static_assert(R == 8, "twiddled butterflies of radix 2, 4, 8");
    // dft<8>'s split: the 4-point DFTs of the even and of the odd inputs
    const T h = (T)0.70710678118654752440;  // sqrt(2)/2
    C e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6];
    dft4_tw<T, C>(e0, e1, e2, e3, w[2], w[4], w[6]);
    C o0 = cmul(u[1], w[1]), o1 = u[3], o2 = u[5], o3 = u[7];
    dft4_tw<T, C>(o0, o1, o2, o3, w[3], w[5], w[7]);
    const C v1 = C{h * (o1.x + o1.y), h * (o1.y - o1.x)};
    const C v2 = mul_mi(o2);
    const C v3 = C{h * (o3.y - o3.x), -h * (o3.x + o3.y)};
    u[0] = cadd(e0, o0);
    u[4] = csub(e0, o0);
    u[1] = cadd(e1, v1);
    u[5] = csub(e1, v1);
    u[2] = cadd(e2, v2);
    u[6] = csub(e2, v2);
    u[3] = cadd(e3, v3);
    u[7] = csub(e3, v3);
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
    if constexpr (sizeof(T) == 8 && R != 3) {
      if (ps > 1) {
        const int step = k * tstride;
        C w[R];
        w[0] = C{(T)1, (T)0};
#pragma unroll
        for (int q = 1; q < R; ++q) w[q] = tw[q * step];
        dft_tw<T, C, R>(u, w);
      } else {
        dft<T, C, R>(u);
      }
    } else {
      if (ps > 1) {
        const int step = k * tstride;
#pragma unroll
        for (int q = 1; q < R; ++q) u[q] = cmul(u[q], tw[q * step]);
      }
      dft<T, C, R>(u);
    }
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

enum LoadMode { LD_PLAIN = 0, LD_RESID = 1 };
enum StoreMode { SO_PLAIN = 0, SO_PCG = 1 };

// Operands of one tile: fields, PCG scalars and tile shape.
template <typename T>
struct DhtTile {
  const T *in;
  T *out;
  T *r;
  const T *q;
  T *p;
  T *x;
  T alpha, beta;
  int first;
  int logP;
};

// Hartley value pairs of outputs m and N - m from X = X_m and Y = X_{N-m}:
// hk = (X.x - X.y + Y.x + Y.y, X.x + X.y - Y.x + Y.y) and hm the same with X and
// Y swapped, from four shared sums (8 adds instead of 12). X = Y (a
// self-paired output) gives hk = hm = 2 X.
template <typename C>
__device__ __forceinline__ void hartley_both(const C X, const C Y, C &hk, C &hm) {
  const auto u = X.x + Y.x, v = X.y - Y.y, w = X.x - Y.x, z = X.y + Y.y;
  hk = C{u - v, w + z};
  hm = C{u + v, z - w};
}

// Shared-memory layout: two ping-pong buffers of N (P+1) complex values, N
// twiddles, then rank x 2P column factors (pass C with a rank-R tensor).
template <typename T>
__host__ __device__ inline size_t dht_smem_bytes_t(int N, int P, int rank) {
  const size_t c = 2 * sizeof(T);
  return 2 * (size_t)N * (P + 1) * c + (size_t)N * c + (size_t)rank * 2 * P * sizeof(T);
}

// Routes of the x2 / x1 tiles (see dht.cu):
//   XF_HARTLEY: Hartley transforms throughout (x2: FFT + Hartley combine);
//   XF_FWD / XF_INV (x2, the complex route): the FFT of the packed pair, no
//     combine; XF_INV stores output j from FFT index N - j, i.e. the inverse
//     transform F* V = F V (-j), up to N;
//   XF_MIRROR (x1 with SCALE): pass C of the complex route. Its input is the
//     x2 spectrum Z(., k2) of packed pairs (a + i b), so the mirror of mode
//     (k1, k2) is (N - k1, N - k2): a tile holds rows k2 and N - k2 (P/2
//     pencils each, the same x3 columns), or P pencils of one of the
//     self-mirrored rows 0 and N/2. The multiplier enters as 8 G: the two x2
//     Hartley combines this route drops each carried a factor 2.
enum DhtRoute { XF_HARTLEY = 0, XF_FWD = 1, XF_INV = 2, XF_MIRROR = 3 };

// One tile: load (with the fused residual update), transform(s), store (with
// the fused PCG update). Per-thread sums of ||r||^2 (LD_RESID) or r.z (SCALE)
// go to acc. Starts with a barrier so consecutive tiles may reuse the buffers.
template <typename T, int AXIS, int LOADM, int STOREM, bool SCALE, int XF = XF_HARTLEY>
__device__ __forceinline__ void dht_tile(const SpectralDev &sp, const DhtTile<T> &a, int tile,
                                         typename Cx<T>::type *buf0, typename Cx<T>::type *buf1,
                                         const typename Cx<T>::type *tw, T *vtab, Accum<T> &acc) {
  static_assert(XF == XF_HARTLEY || (XF == XF_MIRROR) == (AXIS == 1 && SCALE), "route and pass disagree");
  static_assert(XF != XF_MIRROR || sizeof(T) == 8, "the complex route is the FP64 one (its table holds 8 G)");
  static_assert((XF != XF_FWD && XF != XF_INV) || AXIS == 2, "the complex x2 transforms");
  using C = typename Cx<T>::type;
  const int N = sp.N;
  const int logP = a.logP;
  const int P = 1 << logP;
  const int SP = P + 1;
  const int tid = threadIdx.x;
  const size_t NN = (size_t)N * N;
  const int nb2 = N / (2 * P);  // tiles per line for x1 / x2 passes
  const T alpha = a.alpha, beta = a.beta;
  const T *lam = reinterpret_cast<const T *>(sp.lam);
  const T *uf = reinterpret_cast<const T *>(sp.u);
  const int R = sp.rank;
  // pass C works with 2 G (Hartley route) or 8 G (complex route), as the tables hold it
  const T gfac = (XF == XF_MIRROR) ? (T)8 : (T)2;
  const T gscale = gfac * (T)sp.scale;

  __syncthreads();
  // ------------------------------------------------------------------ load
  size_t base = 0, stride = 0;
  int k2 = 0, c0 = 0;
  int rowA = 0, rowB = 0, colA = 0, colB = 0;  // XF_MIRROR: the tile's two halves
  bool pair = false;                            // XF_MIRROR: rows k2 and N - k2
  // x1 / x2 tiles: pencil p (a complex pair of x3 columns) starts at
  // pencil_base(p), its x3 column (the Hartley index k3 of its real part) is
  // pencil_col(p)
  auto pencil_col = [&](int p) -> int {
    if (XF != XF_MIRROR) return c0 + 2 * p;
    const int hp = P >> 1;
    return (p < hp) ? colA + 2 * p : colB + 2 * (p - hp);
  };
  auto pencil_base = [&](int p) -> size_t {
    if (XF != XF_MIRROR) return base + 2 * p;
    const int hp = P >> 1;
    return (p < hp) ? (size_t)rowA * N + colA + 2 * p : (size_t)rowB * N + colB + 2 * (p - hp);
  };
  if (AXIS == 3) {
    const size_t row0 = (size_t)tile * 2 * P;
    const int halfN = N >> 1;
    for (int e = tid; e < P * N; e += kThreads) {
      const int q = e / halfN;
      const int jj = 2 * (e - q * halfN);
      const size_t g = (row0 + q) * N + jj;
      C v = reinterpret_cast<const C *>(a.in)[g >> 1];
      if (LOADM == LD_RESID && !a.first) {
        const C qq = reinterpret_cast<const C *>(a.q)[g >> 1];
        v.x = fma(-alpha, qq.x, v.x);
        v.y = fma(-alpha, qq.y, v.y);
        reinterpret_cast<C *>(a.r)[g >> 1] = v;
        acc.add(fma(v.x, v.x, v.y * v.y));
      }
      T *bs = reinterpret_cast<T *>(buf0);
      bs[(jj * SP + (q >> 1)) * 2 + (q & 1)] = v.x;
      bs[((jj + 1) * SP + (q >> 1)) * 2 + (q & 1)] = v.y;
    }
  } else {
    if (XF == XF_MIRROR) {
      const int tpg = N / P;  // tiles per group: a row pair, or the two self-mirrored rows
      const int gi = tile / tpg, cb = tile - gi * tpg;
      if (gi == 0) {  // rows 0 and N/2, P pencils of one row per tile
        const int hr = tpg >> 1;
        rowA = (cb < hr) ? 0 : (N >> 1);
        colA = ((cb < hr) ? cb : cb - hr) * 2 * P;
        rowB = rowA;
        colB = colA + P;
      } else {  // rows k2 and N - k2, P/2 pencils each
        pair = true;
        rowA = gi;
        rowB = N - gi;
        colA = colB = cb * P;
      }
      k2 = rowA;
      c0 = colA;
      stride = NN;
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
    }
    for (int e = tid; e < P * N; e += kThreads) {
      const int p = e & (P - 1);
      const int j = e >> logP;
      const size_t g = pencil_base(p) + (size_t)j * stride;
      buf0[j * SP + p] = reinterpret_cast<const C *>(a.in)[g >> 1];
    }
    if (SCALE && R > 0 && !sp.gtab) {
      // x2 factors at uf + R N, x3 factors at uf + 2 R N (see SpectralDev);
      // entry 2p + b: pencil p's x3 column b (G, times gfac)
      const T *u2 = uf + (size_t)R * N, *u3 = uf + 2 * (size_t)R * N;
      for (int e = tid; e < R * 2 * P; e += kThreads) {
        const int rr = e / (2 * P), w = e - rr * 2 * P;
        vtab[e] = gfac * (u2[rr * N + k2] * u3[rr * N + pencil_col(w >> 1) + (w & 1)]);
      }
    }
  }
  __syncthreads();
  // --------------------------------------------------------- transform(s)
  C *res = fft_all<T, C>(buf0, buf1, tw, sp, SP, logP);
  // the multiplier at modes (k, k2, k3a) and (k, k2, k3a + 1), k3a = pencil_col(p),
  // times gfac (G(k) = G(N - k) in every index)
  auto multiplier = [&](int k, int p, T &ga, T &gb) {
    const int k3a = pencil_col(p), k3b = k3a + 1;
    if (sp.gtab) {  // tabulated (FP64 (m1, m2, m3), FP32 (m1, m2, k3))
      const int H = (N >> 1) + 1;
      const T *tab = reinterpret_cast<const T *>(sp.gtab);
      if (sizeof(T) == 8) {
        const T *row = tab + ((size_t)mirror_index(k, N) * H + mirror_index(k2, N)) * H;
        ga = row[mirror_index(k3a, N)];
        gb = row[mirror_index(k3b, N)];
      } else {
        const T *row = tab + ((size_t)mirror_index(k, N) * H + mirror_index(k2, N)) * N;
        ga = (k == 0 && k2 == 0 && k3a == 0) ? (T)0 : row[k3a];
        gb = row[k3b];
      }
    } else if (R == 0) {
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
  };
  // Pass C's scaling (described at s2_combine) of the mode pair X = Z(k),
  // Y = Z(mirror of k), in place as conj(W) for the second transform; ga, gb
  // are gfac G. The pair's share of r.z, G_a |X + conj Y|^2 + G_b |X - conj Y|^2
  // in units of the route's factor, equals Re(conj X W_X) + Re(conj Y W_Y)
  // (W_X = s4 X + d4 conj Y, W_Y = s4 Y + d4 conj X: both sides are
  // s4 (|X|^2 + |Y|^2) + 2 d4 Re(X Y)), so it is summed from the scaled values,
  // two FMAs per mode. A self-mirrored mode (Y = X) counts once.
  auto scale_pair = [&](C *px, C *py, bool self, T ga, T gb) {
    const C X = *px, Y = *py;
    const T s4 = ga + gb, d4 = ga - gb;
    const C cwx = C{fma(s4, X.x, d4 * Y.x), fma(d4, Y.y, -s4 * X.y)};  // conj(W_X)
    *px = cwx;
    acc.add_prod(X.x, cwx.x);
    acc.add_prod(-X.y, cwx.y);
    if (!self) {
      const C cwy = C{fma(s4, Y.x, d4 * X.x), fma(d4, X.y, -s4 * Y.y)};
      *py = cwy;
      acc.add_prod(Y.x, cwy.x);
      acc.add_prod(-Y.y, cwy.y);
    }
  };
  if (XF == XF_MIRROR && pair) {
    // rows k2 (pencils p < P/2) and N - k2 (pencil p + P/2): Z(k, k2) pairs
    // with Z(N - k, N - k2), every k, and the two modes always differ
    const int hp = P >> 1;
    for (int t = tid; t < (N << (logP - 1)); t += kThreads) {
      const int p = t & (hp - 1);
      const int k = t >> (logP - 1);
      const int km = (k == 0) ? 0 : N - k;
      T ga, gb;
      multiplier(k, p, ga, gb);
      scale_pair(&res[k * SP + p], &res[km * SP + p + hp], false, ga, gb);
    }
    __syncthreads();
  } else if (SCALE || XF == XF_HARTLEY) {
    const int halfN = N >> 1;
    for (int t = tid; t < ((halfN + 1) << logP); t += kThreads) {
      const int p = t & (P - 1);
      const int k = t >> logP;
      const int km = (k == 0) ? 0 : N - k;
      if (SCALE) {
        T ga, gb;
        multiplier(k, p, ga, gb);
        scale_pair(&res[k * SP + p], &res[km * SP + p], km == k, ga, gb);
      } else {
        const C X = res[k * SP + p], Y = res[km * SP + p];
        C hk, hm;
        hartley_both(X, Y, hk, hm);
        res[k * SP + p] = hk;
        if (km != k) res[km * SP + p] = hm;
      }
    }
    __syncthreads();
  }
  if (SCALE) {  // the inverse: forward transform of conj(W), stored conjugated (below)
    C *other = (res == buf0) ? buf1 : buf0;
    res = fft_all<T, C>(res, other, tw, sp, SP, logP);
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
      const size_t g = pencil_base(p) + (size_t)j * stride;
      const int js = (XF == XF_INV && j != 0) ? N - j : j;
      const C v = res[js * SP + p];
      reinterpret_cast<C *>(a.out)[g >> 1] = SCALE ? C{v.x, -v.y} : v;
    }
  }
}

}  // namespace sq

namespace sq {

// ----------------------------------------------------------------------------
// Two-stage tiles (FP32): N = R0 * R1 with radices 3, 4, 6, 8, 16, 32, P complex
// pencils per tile, all shape parameters compile-time so that the index
// arithmetic folds to shifts and constants. One shared-memory round trip per
// transform.
//
// Strided axes (x1, x2): pencil p of a tile is the complex column 2P-wide row
// segment element p; shared memory holds position j of pencil p at j SP + p,
// SP = P + 1.
//   stage 1 (radix R0, no twiddles): butterfly b < R1 of pencil p reads
//     x[b + q R1] (q < R0) -- from global memory (rows of P complex values,
//     coalesced) or from shared memory (second transform of pass C) -- and
//     writes y[b R0 + q] to shared memory;
//   stage 2 (radix R1, last): butterfly b < R0 reads y[b + q R0], applies
//     tw[q b], and yields X[b + q R0] in place (a butterfly reads and writes
//     only its own positions, so no barrier is needed inside the stage);
//   combine: thread (p, k), k <= N/2, forms the Hartley values 2(H a), 2(H b)
//     at k and N - k and stores them (pass C: scales by G, reduces r.z and
//     writes them back for the second transform).
// ----------------------------------------------------------------------------
constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

template <typename T, typename C, int R0, int R1, int P, bool FROM_SMEM, long long STRIDE>
__device__ __forceinline__ void s2_stage1(const C *__restrict__ gsrc, size_t base, C *sm) {
  constexpr int SP = P + 1, LP = ilog2c(P);
  static_assert(R1 * P <= kThreads, "one stage-1 butterfly per thread");
  const int t = threadIdx.x;
  const int p = t & (P - 1), b = t >> LP;
  C u[R0];
  if (t < R1 * P) {
    const C *g = gsrc + (base >> 1) + (size_t)b * (STRIDE >> 1) + p;
#pragma unroll
    for (int q = 0; q < R0; ++q) u[q] = FROM_SMEM ? sm[(b + q * R1) * SP + p] : g[(size_t)q * R1 * (STRIDE >> 1)];
    dft<T, C, R0>(u);
  }
  if (FROM_SMEM) __syncthreads();  // every read of the tile precedes the overwrite
  if (t < R1 * P) {
#pragma unroll
    for (int q = 0; q < R0; ++q) sm[(b * R0 + q) * SP + p] = u[q];
  }
  __syncthreads();
}


// (R0 P may exceed the block: a thread then takes several butterflies, each
// reading and writing only its own positions.)
template <typename T, typename C, int R0, int R1, int P>
__device__ __forceinline__ void s2_stage2(C *sm, const C *__restrict__ tw) {
  constexpr int SP = P + 1, LP = ilog2c(P);
  for (int t = threadIdx.x; t < R0 * P; t += kThreads) {
    const int p = t & (P - 1), b = t >> LP;
    C x[R1];
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      x[q] = sm[(b + q * R0) * SP + p];
      if (q > 0) x[q] = cmul(x[q], tw[q * b]);
    }
    dft<T, C, R1>(x);
#pragma unroll
    for (int q = 0; q < R1; ++q) sm[(b + q * R0) * SP + p] = x[q];
  }
  __syncthreads();
}

// Multiplier G at (k, k2, k3a) and (k, k2, k3a + 1), k3a = c0 + 2p: exact
// (RR = 0), rank RR with the column factors va/vb of this thread's pencil in
// registers (RR > 0), a runtime rank (RR = -1, factors read from vtab), or
// read from the tile's slice of the FP32 multiplier table that dht_tile_s2
// prefetched into vtab (RR = -2: row k <= N/2, the tile's 2P columns). Every
// form yields 2 G, as the tables hold it (the factor is exact).
template <typename T, int N, int P, int RR>
__device__ __forceinline__ void s2_multiplier(const SpectralDev &sp, int k, int k2, int c0, int p, const T *vtab,
                                              const T (&va)[RR > 0 ? RR : 1], const T (&vb)[RR > 0 ? RR : 1],
                                              T gscale, T &ga, T &gb) {
  const T *lam = reinterpret_cast<const T *>(sp.lam);
  const T *uf = reinterpret_cast<const T *>(sp.u);
  const int k3a = c0 + 2 * p;
  if constexpr (RR == -2) {
    const T *tt = vtab + (size_t)k * 2 * P + 2 * p;
    ga = (k == 0 && k2 == 0 && k3a == 0) ? (T)0 : tt[0];
    gb = tt[1];
  } else if constexpr (RR == 0) {  // gscale: 2 / (64 N^3), in T
    const T l12 = lam[k] + lam[k2];
    const T g1 = l12 + lam[k3a], g2 = l12 + lam[k3a + 1];
    ga = (g1 > (T)0) ? gscale / g1 : (T)0;
    gb = (g2 > (T)0) ? gscale / g2 : (T)0;
  } else {
    T sa = (T)0, sb = (T)0;
    if constexpr (RR > 0) {
#pragma unroll
      for (int rr = 0; rr < RR; ++rr) {
        const T uk = uf[rr * N + k];
        sa = fma(uk, va[rr], sa);
        sb = fma(uk, vb[rr], sb);
      }
    } else {
      for (int rr = 0; rr < sp.rank; ++rr) {
        const T uk = uf[rr * N + k];
        sa = fma(uk, vtab[rr * 2 * P + 2 * p], sa);
        sb = fma(uk, vtab[rr * 2 * P + 2 * p + 1], sb);
      }
    }
    ga = (k == 0 && k2 == 0 && k3a == 0) ? (T)0 : sa;
    gb = sb;  // k3a + 1 >= 1
  }
}

// Pass C scales in the Fourier domain. Along x1 the multiplier g is even
// (g(k) = g(N-k)), so H diag(g) H = F* diag(g) F: with the two real pencils
// a, b of a complex pencil, Z = F(a + ib), A = F a = (Z_k + conj Z_{N-k}) / 2
// and B = F b = (Z_k - conj Z_{N-k}) / 2i, the scaled spectrum is
//   W_k = g_a A_k + i g_b B_k = s Z_k + d conj(Z_{N-k}),
//   s = (g_a + g_b) / 2, d = (g_a - g_b) / 2,
// and F*(W) = conj(F(conj W)) has the results for a and b as its real and
// imaginary parts: the inverse is the forward transform of conj(W), stored
// conjugated, with no Hartley combine on either side. The factor 4 of the
// two Hartley combines this replaces is folded into s and d: the multiplier
// arrives as 2 G, so 4 s = 2G_a + 2G_b and 4 d = 2G_a - 2G_b with no further
// product. r.z (Parseval): g_a |A_k|^2 + g_b |B_k|^2 per k.
// s2_combine MODE 0: Hartley combine, store to global (rows of P complex
// values, coalesced); 1: pass C's scaling above, reduce r.z into acc, write
// conj(W) back in place for the second transform; 2: store the conjugate.
template <typename T, typename C, int N, int P, int MODE, int RR, long long STRIDE>
__device__ __forceinline__ void s2_combine(C *sm, C *__restrict__ gdst, size_t base, const SpectralDev &sp, int k2,
                                           int c0, const T *vtab, Accum<T> &acc) {
  constexpr int SP = P + 1, LP = ilog2c(P);
  const int p = threadIdx.x & (P - 1);  // the same pencil for all of this thread's outputs
  T va[RR > 0 ? RR : 1], vb[RR > 0 ? RR : 1];
  if constexpr (MODE == 1 && RR > 0) {
#pragma unroll
    for (int rr = 0; rr < RR; ++rr) {
      va[rr] = vtab[rr * 2 * P + 2 * p];
      vb[rr] = vtab[rr * 2 * P + 2 * p + 1];
    }
  }
  C *g = gdst + (base >> 1) + p;
  const T gscale = (T)2 * (T)sp.scale;  // converted once, outside the loop (the FP64 pipe is narrow)
  for (int t = threadIdx.x; t < ((N / 2 + 1) << LP); t += kThreads) {
    const int k = t >> LP;
    const int km = (k == 0) ? 0 : N - k;
    const C X = sm[k * SP + p], Y = sm[km * SP + p];
    if (MODE == 1) {
      T ga, gb;
      s2_multiplier<T, N, P, RR>(sp, k, k2, c0, p, vtab, va, vb, gscale, ga, gb);  // G(N - k) = G(k)
      // ga, gb are 2 G: e2 below is already doubled, the share of both modes k, N - k
      const T sx = X.x + Y.x, dy = X.y - Y.y, dx = X.x - Y.x, sy = X.y + Y.y;
      T e2 = fma(ga, fma(sx, sx, dy * dy), gb * fma(dx, dx, sy * sy));
      if (km == k) e2 *= (T)0.5;
      acc.add(e2);
      const T s4 = ga + gb, d4 = ga - gb;
      sm[k * SP + p] = C{fma(s4, X.x, d4 * Y.x), fma(d4, Y.y, -s4 * X.y)};
      if (km != k) sm[km * SP + p] = C{fma(s4, Y.x, d4 * X.x), fma(d4, X.y, -s4 * Y.y)};
    } else if (MODE == 2) {
      g[(size_t)k * (STRIDE >> 1)] = C{X.x, -X.y};
      if (km != k) g[(size_t)km * (STRIDE >> 1)] = C{Y.x, -Y.y};
    } else {
      C hk, hm;
      hartley_both(X, Y, hk, hm);
      g[(size_t)k * (STRIDE >> 1)] = hk;
      if (km != k) g[(size_t)km * (STRIDE >> 1)] = hm;
    }
  }
  __syncthreads();
}

// Strided-axis tile (AXIS 1 or 2) with the two-stage plan R0 x R1. SCALE: pass C.
template <typename T, int AXIS, int R0, int R1, int P, bool SCALE, int RR>
__device__ __forceinline__ void dht_tile_s2(const SpectralDev &sp, const DhtTile<T> &a, int tile,
                                            typename Cx<T>::type *sm, const typename Cx<T>::type *tw, T *vtab,
                                            Accum<T> &acc) {
  using C = typename Cx<T>::type;
  constexpr int N = R0 * R1;
  constexpr long long NN = (long long)N * N;
  constexpr long long STRIDE = (AXIS == 2) ? N : NN;
  constexpr int nb2 = N / (2 * P);
  static_assert(nb2 >= 1, "a tile of 2P pencils must fit the grid");
  const int line = tile / nb2, cb = tile - line * nb2;
  const int c0 = cb * 2 * P;
  const size_t base = (AXIS == 2) ? (size_t)line * NN + c0 : (size_t)line * N + c0;
  const int k2 = line;
  __syncthreads();
  if constexpr (SCALE && RR == -2) {
    // the tile's slice of the multiplier table, rows m1 = 0..N/2 of its 2P
    // columns at (m2 = mirror(k2), k3 = c0 ..), fetched while the first
    // transform runs (16-byte cp.async; waited for before stage 2)
    constexpr int H = N / 2 + 1, CH = 2 * P / 4;
    const T *gt = reinterpret_cast<const T *>(sp.gtab) + (size_t)mirror_index(k2, N) * N + c0;
    for (int e = threadIdx.x; e < H * CH; e += kThreads) {
      const int m1 = e / CH, ch = e - m1 * CH;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(vtab + (size_t)m1 * 2 * P + 4 * ch);
      const T *src = gt + (size_t)m1 * H * N + 4 * ch;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  if (SCALE && RR != 0 && RR != -2) {
    const T *uf = reinterpret_cast<const T *>(sp.u);
    const T *u2 = uf + (size_t)sp.rank * N, *u3 = uf + 2 * (size_t)sp.rank * N;  // x2, x3 factors
    for (int e = threadIdx.x; e < sp.rank * 2 * P; e += kThreads) {
      const int rr = e / (2 * P), w = e - rr * 2 * P;
      vtab[e] = (T)2 * (u2[rr * N + k2] * u3[rr * N + c0 + w]);  // 2 G, as the tables hold it
    }
  }
  const C *gin = reinterpret_cast<const C *>(a.in);
  C *gout = reinterpret_cast<C *>(a.out);
  s2_stage1<T, C, R0, R1, P, false, STRIDE>(gin, base, sm);
  if constexpr (SCALE && RR == -2) asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // stage 2 ends with a barrier
  s2_stage2<T, C, R0, R1, P>(sm, tw);
  if (SCALE) {
    s2_combine<T, C, N, P, 1, RR, STRIDE>(sm, gout, base, sp, k2, c0, vtab, acc);
    s2_stage1<T, C, R0, R1, P, true, STRIDE>(gin, base, sm);
    s2_stage2<T, C, R0, R1, P>(sm, tw);
    s2_combine<T, C, N, P, 2, RR, STRIDE>(sm, gout, base, sp, k2, c0, vtab, acc);
  } else {
    s2_combine<T, C, N, P, 0, RR, STRIDE>(sm, gout, base, sp, k2, c0, vtab, acc);
  }
}

// ----------------------------------------------------------------------------
// Two-stage tile for the contiguous axis (x3): 2P consecutive rows of N reals,
// rows 2p and 2p+1 forming complex pencil p. Shared memory holds pencil p at
// p * SJ + x3pos(j) with one pad entry per 16 (SJ = x3pos(N)), so that the
// stage-1 writes (stride R0 = 16 along j across lanes) and the stage-2 /
// combine accesses (consecutive j across lanes) are conflict-free.
//   stage 1: butterfly (p, b), b < R1, b fastest so that lanes read
//     consecutive row entries: x[b + q R1] of rows 2p, 2p+1 for q < R0 (pass
//     A fuses r -= alpha q and ||r||^2 here), radix R0, y -> x3pos(b R0 + q);
//   stage 2: butterfly (p, b), b < R0, in place on x3pos(b + q R0): twiddles
//     tw[q b], radix R1, giving X[b + q R0];
//   combine: (p, k), 0 < k < N/2, forms the Hartley values of both rows at k
//     and N - k (k = 0 also takes the self-paired 0 and N/2) and stores them
//     along the rows (pass E fuses x += alpha p, p = z + beta p).
// ----------------------------------------------------------------------------
__host__ __device__ constexpr int x3pos(int j) { return j + (j >> 4); }

// The fields a kernel reads and writes may alias (pass A reads r through
// `in` and writes it through `r`), so the compiler keeps every load behind
// the stores before it; each butterfly therefore issues its loads in chunks
// of HC pairs ahead of the chunk's stores, one memory latency per chunk.
template <typename T, typename C, int R0, int R1, int P, int LOADM>
__device__ __forceinline__ void x3_stage1(const DhtTile<T> &a, size_t row0, C *sm, Accum<T> &acc) {
  constexpr int N = R0 * R1;
  constexpr int SJ = x3pos(N);
  constexpr int HC = R0 > 8 ? 8 : R0;
  const T alpha = a.alpha;
  // With the residual update r is read and written through one pointer (the
  // offsets of a butterfly's chunks are distinct constants, so the compiler
  // may issue a chunk's loads ahead of the previous chunk's stores), and q,
  // which nothing writes during the pass, through a restricted one.
  const bool resid = LOADM == LD_RESID && !a.first;
  const T *inp = resid ? a.r : a.in;
  const T *__restrict__ qp = a.q;
  for (int t = threadIdx.x; t < R1 * P; t += kThreads) {
    const int p = t / R1, b = t - p * R1;
    const size_t ga = (row0 + 2 * p) * N + b, gb = ga + N;
    C u[R0];
#pragma unroll
    for (int h = 0; h < R0; h += HC) {
      T va[HC], vb[HC];
#pragma unroll
      for (int q = 0; q < HC; ++q) {
        va[q] = inp[ga + (h + q) * R1];
        vb[q] = inp[gb + (h + q) * R1];
      }
      if (LOADM == LD_RESID && !a.first) {
        T qa[HC], qb[HC];
#pragma unroll
        for (int q = 0; q < HC; ++q) {
          qa[q] = qp[ga + (h + q) * R1];
          qb[q] = qp[gb + (h + q) * R1];
        }
#pragma unroll
        for (int q = 0; q < HC; ++q) {
          va[q] = fma(-alpha, qa[q], va[q]);
          vb[q] = fma(-alpha, qb[q], vb[q]);
          acc.add(fma(va[q], va[q], vb[q] * vb[q]));
        }
#pragma unroll
        for (int q = 0; q < HC; ++q) {
          a.r[ga + (h + q) * R1] = va[q];
          a.r[gb + (h + q) * R1] = vb[q];
        }
      }
#pragma unroll
      for (int q = 0; q < HC; ++q) u[h + q] = C{va[q], vb[q]};
    }
    dft<T, C, R0>(u);
    C *sp = sm + p * SJ;
#pragma unroll
    for (int q = 0; q < R0; ++q) sp[x3pos(b * R0 + q)] = u[q];
  }
  __syncthreads();
}

template <typename T, typename C, int R0, int R1, int P>
__device__ __forceinline__ void x3_stage2(C *sm, const C *__restrict__ tw) {
  constexpr int SJ = x3pos(R0 * R1);
  for (int t = threadIdx.x; t < R0 * P; t += kThreads) {
    const int p = t / R0, b = t - p * R0;
    C *sp = sm + p * SJ;
    C x[R1];
#pragma unroll
    for (int q = 0; q < R1; ++q) {
      x[q] = sp[x3pos(b + q * R0)];
      if (q > 0) x[q] = cmul(x[q], tw[q * b]);
    }
    dft<T, C, R1>(x);
#pragma unroll
    for (int q = 0; q < R1; ++q) sp[x3pos(b + q * R0)] = x[q];
  }
  __syncthreads();
}

// ------------------------------------------------- bulk copies (sm_90+)
// One-dimensional global -> shared copies by the asynchronous copy engine,
// completing on a shared-memory mbarrier (transaction count in bytes).
// Addresses and sizes must be multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Arms the barrier's current phase for `bytes` and issues the copy (one thread).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
// Waits, at most max_tries polls, for the phase of parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, unsigned parity, int max_tries) {
  for (int i = 0; i < max_tries; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Stores the values v[0..3] of row positions g[0..3]: plain, or the fused PCG
// update (all loads of the four positions before any store; see x3_stage1).
// pl / xl: the tile's p and x rows staged in shared memory (element g at
// g - base), or null to read them from global memory.
template <typename T, int STOREM>
__device__ __forceinline__ void x3_put4(const DhtTile<T> &a, const size_t (&g)[4], const T (&v)[4],
                                        const T *pl = nullptr, const T *xl = nullptr, size_t base = 0) {
  if (STOREM == SO_PCG) {
    if (a.first) {
#pragma unroll
      for (int i = 0; i < 4; ++i) a.p[g[i]] = v[i];
    } else {
      T po[4], xo[4];
      if (pl) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          po[i] = pl[g[i] - base];
          xo[i] = xl[g[i] - base];
        }
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          po[i] = a.p[g[i]];
          xo[i] = a.x[g[i]];
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a.x[g[i]] = fma(a.alpha, po[i], xo[i]);
        a.p[g[i]] = fma(a.beta, po[i], v[i]);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) a.out[g[i]] = v[i];
  }
}

template <typename T, typename C, int N, int P, int STOREM>
__device__ __forceinline__ void x3_combine(const DhtTile<T> &a, size_t row0, const C *sm, const T *pl = nullptr,
                                           const T *xl = nullptr) {
  constexpr int H = N / 2;
  constexpr int SJ = x3pos(N);
  for (int t = threadIdx.x; t < H * P; t += kThreads) {
    const int p = t / H, k = t - p * H;
    const C *sp = sm + p * SJ;
    const size_t ga = (row0 + 2 * p) * N, gb = ga + N;
    const int km = (k == 0) ? H : N - k;  // k = 0: the second self-paired output is N/2
    const C X = sp[x3pos(k)], Y = sp[x3pos(km)];
    // k = 0: outputs 0 and N/2 are their own mirrors (2 X and 2 Y)
    C hk, hm;
    hartley_both(X, k == 0 ? X : Y, hk, hm);
    if (k == 0) hm = C{Y.x + Y.x, Y.y + Y.y};
    const size_t g[4] = {ga + k, gb + k, ga + km, gb + km};
    const T v[4] = {hk.x, hk.y, hm.x, hm.y};
    x3_put4<T, STOREM>(a, g, v, pl, xl, row0 * N);
  }
}

}  // namespace sq
