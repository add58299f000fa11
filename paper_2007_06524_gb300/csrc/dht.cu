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
//      sum_r u1_r u2_r u3_r), reduce r.z, x1 transform again, in place; the
//      scaling acts on the complex spectrum directly and the inverse is the
//      conjugated forward transform (no Hartley combine; see s2_combine)
//   D: x2 transform, in place
//   E: x3 transform -> z (PCG: x += alpha p; p = z + beta p)
// A tile is P complex pencils = 2P real pencils: 2P adjacent rows for x3,
// 2P adjacent x3-columns for x1 and x2 (coalesced 2P-wide row segments).
//
// FP64 takes a complex route through B, C and D. G is even in k2 too, so
// the x2 Hartley pair around pass C equals F2* (.) F2: B stores the FFT of
// each packed pair a + i b (two x3 Hartley columns) with no combine, D the
// inverse (the forward FFT read from index N - j). Pass C then sees
// Z(k1, k2) = A + i B with A, B the 2D FFTs of the real a, b, whose mirror
// mode is (N - k1, N - k2): its tiles hold rows k2 and N - k2 together (rows
// 0 and N/2 pair within themselves), and the scaling above applies unchanged
// with the multiplier as 8 G (the two dropped combines each carried a factor
// 2). The fields keep the same real layout in HBM; passes A and E keep their
// combines, since the rows they pack are mixed by the later transforms.
#include "dht_core.cuh"

namespace sq {

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
  int stage;  // pass E with the PCG update: stage the tile's p and x rows (set by the launcher)
  int wait_polls;  // polls of a staging wait before it gives up (set by the launcher)
};

template <typename T, int AXIS, int LOADM, int STOREM, bool SCALE, int XF = XF_HARTLEY>
__global__ void __launch_bounds__(kThreads) k_dht(DhtArgs<T> a) {
  using C = typename Cx<T>::type;
  if (a.check_done && *(volatile int *)&a.rb.st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.sp.N;
  const int P = 1 << a.logP;
  C *buf0 = reinterpret_cast<C *>(smem_raw);
  C *buf1 = buf0 + N * (P + 1);
  C *tw = buf1 + N * (P + 1);
  T *vtab = reinterpret_cast<T *>(tw + N);
  const C *twg = reinterpret_cast<const C *>(a.sp.tw);
  for (int m = threadIdx.x; m < N; m += kThreads) tw[m] = twg[m];
  DhtTile<T> t;
  t.in = a.in;
  t.out = a.out;
  t.r = a.r;
  t.q = a.q;
  t.p = a.p;
  t.x = a.x;
  t.alpha = (T)a.rb.st->alpha;
  t.beta = (T)a.rb.st->beta;
  t.first = a.first;
  t.logP = a.logP;
  Accum<T> acc;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x)
    dht_tile<T, AXIS, LOADM, STOREM, SCALE, XF>(a.sp, t, tile, buf0, buf1, tw, vtab, acc);
  if (LOADM == LD_RESID || SCALE) {
    typename Accum<T>::Part v[1] = {acc.part()};
    double s[1];
    if (reduce_last_block<1>(v, a.rb.partials, &a.rb.st->ticket, s)) {
      if (threadIdx.x == 0) {
        int op = FIN_NONE;
        if (LOADM == LD_RESID) op = a.first ? FIN_NONE : FIN_RR_ITER;
        if (SCALE) op = a.first ? FIN_RZ_FIRST : FIN_RZ_BETA;
        finalize_scalars(a.rb.st, op, s, 1);
      }
    }
  }
}

// Two-stage passes (FP32; see dht_tile_s2 and x3_stage1). A tile holds ~38 KB
// of shared memory at N = 256, P = 16: room for 5 blocks per SM, of which the
// register cap sets how many stay resident. Blocks per SM the cap aims at:
// 4 (64 registers) for passes A to D: A, B and D fit that without spilling,
// and pass C (128 registers uncapped) spills a few words but gains more from
// the fourth block than the spills cost; 3 (80 registers) for pass E, which
// its bulk-copy staging buffers hold to 2 blocks per SM by shared memory
// anyway; 2 for the radix-32 stages of N = 512 (up to 128 registers).
// Strided axes x1 (pass C, SCALE) and x2 (passes B, D).
constexpr int s2_min_blocks(int n, bool cap80) { return n > 256 ? 2 : (cap80 ? 3 : 4); }

template <int AXIS, int R0, int R1, int P, bool SCALE, int RR>
__global__ void __launch_bounds__(kThreads, s2_min_blocks(R0 * R1, false)) k_dht_s2(DhtArgs<float> a) {
  using C = float2;
  if (a.check_done && *(volatile int *)&a.rb.st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int N = R0 * R1;
  C *sm = reinterpret_cast<C *>(smem_raw);
  C *tw = sm + N * (P + 1);
  float *vtab = reinterpret_cast<float *>(tw + N);
  const C *twg = reinterpret_cast<const C *>(a.sp.tw);
  for (int m = threadIdx.x; m < N; m += kThreads) tw[m] = twg[m];
  DhtTile<float> t;
  t.in = a.in;
  t.out = a.out;
  t.r = a.r;
  t.q = a.q;
  t.p = a.p;
  t.x = a.x;
  t.alpha = (float)a.rb.st->alpha;
  t.beta = (float)a.rb.st->beta;
  t.first = a.first;
  t.logP = a.logP;
  Accum<float> acc;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x)
    dht_tile_s2<float, AXIS, R0, R1, P, SCALE, RR>(a.sp, t, tile, sm, tw, vtab, acc);
  if (SCALE) {
    FF v[1] = {acc.part()};
    double s[1];
    if (reduce_last_block<1>(v, a.rb.partials, &a.rb.st->ticket, s)) {
      if (threadIdx.x == 0) finalize_scalars(a.rb.st, a.first ? FIN_RZ_FIRST : FIN_RZ_BETA, s, 1);
    }
  }
}

template <int AXIS, int R0, int R1, int P, bool SCALE, int RR>
static cudaError_t launch_s2(const DhtArgs<float> &a, int grid, cudaStream_t s) {
  const size_t vtab = (RR == -2) ? (size_t)(R0 * R1 / 2 + 1) * 2 * P : (size_t)a.sp.rank * 2 * P;
  const size_t smem = (size_t)R0 * R1 * (P + 1) * sizeof(float2) + (size_t)R0 * R1 * sizeof(float2) +
                      vtab * sizeof(float);
  auto kern = k_dht_s2<AXIS, R0, R1, P, SCALE, RR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Specialisations of pass C: exact (0), the tabulated multiplier (-2, where
// the preconditioner carries one), rank 8 in registers, else runtime.
template <int AXIS, int R0, int R1, int P, bool SCALE>
static cudaError_t launch_s2_rank(const DhtArgs<float> &a, int grid, cudaStream_t s) {
  if constexpr (!SCALE) {
    return launch_s2<AXIS, R0, R1, P, SCALE, -1>(a, grid, s);
  } else {
    // the exact diagonal's divide measured faster than the table's prefetch
    // (51.5 against 52.4 us at N = 256); rank 8 the other way (54.2 against 52.3)
    if (a.sp.rank == 0) return launch_s2<AXIS, R0, R1, P, SCALE, 0>(a, grid, s);
    if (a.sp.gtab) return launch_s2<AXIS, R0, R1, P, SCALE, -2>(a, grid, s);
    if (a.sp.rank == 8) return launch_s2<AXIS, R0, R1, P, SCALE, 8>(a, grid, s);
    return launch_s2<AXIS, R0, R1, P, SCALE, -1>(a, grid, s);
  }
}

// P = 8 or 16 pencils where tiles of 2P pencils cover the grid (2P | N).
template <int AXIS, int R0, int R1, bool SCALE>
static cudaError_t launch_s2_p(const DhtArgs<float> &a, int grid, cudaStream_t s) {
  if constexpr ((R0 * R1) % 16 == 0) {
    if (a.logP == 3) return launch_s2_rank<AXIS, R0, R1, 8, SCALE>(a, grid, s);
  }
  if constexpr ((R0 * R1) % 32 == 0 && R1 * 16 <= kThreads) {
    if (a.logP == 4) return launch_s2_rank<AXIS, R0, R1, 16, SCALE>(a, grid, s);
  }
  return cudaErrorNotSupported;
}

// Two-stage plans for the strided passes; cudaErrorNotSupported when N or P has none.
template <int AXIS, bool SCALE>
static cudaError_t launch_strided_fast(const DhtArgs<float> &a, int grid, cudaStream_t s) {
  switch (a.sp.N) {
    case 16: return launch_s2_p<AXIS, 4, 4, SCALE>(a, grid, s);
    case 32: return launch_s2_p<AXIS, 8, 4, SCALE>(a, grid, s);
    case 48: return launch_s2_p<AXIS, 16, 3, SCALE>(a, grid, s);
    case 64: return launch_s2_p<AXIS, 8, 8, SCALE>(a, grid, s);
    case 96: return launch_s2_p<AXIS, 16, 6, SCALE>(a, grid, s);
    case 128: return launch_s2_p<AXIS, 16, 8, SCALE>(a, grid, s);
    case 256: return launch_s2_p<AXIS, 16, 16, SCALE>(a, grid, s);
    case 512: return launch_s2_p<AXIS, 32, 16, SCALE>(a, grid, s);
    default: return cudaErrorNotSupported;
  }
}

// Contiguous axis x3 (passes A and E).
template <int R0, int R1, int P, int LOADM, int STOREM>
__global__ void __launch_bounds__(kThreads, s2_min_blocks(R0 * R1, STOREM == SO_PCG)) k_dht_s3(DhtArgs<float> a) {
  using C = float2;
  if (a.check_done && *(volatile int *)&a.rb.st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int N = R0 * R1;
  constexpr int SJ = x3pos(N);
  C *sm = reinterpret_cast<C *>(smem_raw);
  C *tw = sm + (size_t)P * SJ;
  const C *twg = reinterpret_cast<const C *>(a.sp.tw);
  for (int m = threadIdx.x; m < N; m += kThreads) tw[m] = twg[m];
  DhtTile<float> t;
  t.in = a.in;
  t.out = a.out;
  t.r = a.r;
  t.q = a.q;
  t.p = a.p;
  t.x = a.x;
  t.alpha = (float)a.rb.st->alpha;
  t.beta = (float)a.rb.st->beta;
  t.first = a.first;
  t.logP = a.logP;
  Accum<float> acc;
  // Pass E with the PCG update: the tile's p and x rows (2P N contiguous
  // floats each) are fetched into shared memory by two bulk copies issued at
  // the start of the tile, so they land while the tile is transformed.
  // Every wait is bounded; a thread whose wait gives up reads global memory
  // and flags the fault, and the block stops staging (that barrier phase
  // never completed and must not be armed again).
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ int s_stage_off;
  float *pl = nullptr, *xl = nullptr;
  bool staged = (STOREM == SO_PCG) && !a.first && a.stage;
  unsigned phase = 0;
  bool late = false;  // a wait gave up: that phase's copies may still be in flight
  if (staged) {
    pl = reinterpret_cast<float *>(tw + N);
    xl = pl + 2 * P * N;
    if (threadIdx.x == 0) {
      mbar_init(&mbar, 1);
      s_stage_off = 0;
    }
  }
  constexpr unsigned kRowBytes = 2u * P * N * sizeof(float);
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    __syncthreads();  // twiddles loaded; the previous tile's combine is done with sm, pl, xl
    if (staged && s_stage_off) staged = false;
    const size_t row0 = (size_t)tile * 2 * P;
    if (staged && threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(&mbar, 2 * kRowBytes);
      bulk_g2s(pl, a.p + row0 * N, kRowBytes, &mbar);
      bulk_g2s(xl, a.x + row0 * N, kRowBytes, &mbar);
    }
    x3_stage1<float, C, R0, R1, P, LOADM>(t, row0, sm, acc);
    x3_stage2<float, C, R0, R1, P>(sm, tw);
    if (staged) {
      const bool ok = mbar_wait(&mbar, phase, a.wait_polls);
      phase ^= 1u;
      if (!ok) {
        a.rb.st->fault = 1;
        s_stage_off = 1;
        late = true;
      }
      x3_combine<float, C, N, P, STOREM>(t, row0, sm, ok ? pl : nullptr, ok ? xl : nullptr);
    } else {
      x3_combine<float, C, N, P, STOREM>(t, row0, sm);
    }
  }
  // do not leave with a copy into this block in flight (this drain keeps its
  // own, long limit whatever the option says)
  if (late) mbar_wait(&mbar, phase ^ 1u, 1 << 24);
  if (LOADM == LD_RESID) {
    FF v[1] = {acc.part()};
    double s[1];
    if (reduce_last_block<1>(v, a.rb.partials, &a.rb.st->ticket, s)) {
      if (threadIdx.x == 0) finalize_scalars(a.rb.st, a.first ? FIN_NONE : FIN_RR_ITER, s, 1);
    }
  }
}


template <int R0, int R1, int P, int LOADM, int STOREM>
static cudaError_t launch_s3(const DhtArgs<float> &a, int grid, cudaStream_t s) {
  // pass E with the PCG update also stages the tile's p and x rows, where the
  // block still fits twice on an SM
  const size_t base = ((size_t)P * x3pos(R0 * R1) + (size_t)R0 * R1) * sizeof(float2);
  const size_t rows = 2 * (size_t)(2 * P * R0 * R1) * sizeof(float);
  DhtArgs<float> b = a;
  // bulk copies need 16-byte aligned rows (the workspace fields are)
  const bool aligned = ((reinterpret_cast<uintptr_t>(a.p) | reinterpret_cast<uintptr_t>(a.x)) & 15) == 0;
  b.stage = (STOREM == SO_PCG && !a.first && aligned && base + rows <= 110 * 1024) ? 1 : 0;
  b.wait_polls = sq::stage_wait_polls();
  const size_t smem = base + (b.stage ? rows : 0);
  auto kern = k_dht_s3<R0, R1, P, LOADM, STOREM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(b);
  return cudaGetLastError();
}

template <int R0, int R1, int LOADM, int STOREM>
static cudaError_t launch_s3_p(const DhtArgs<float> &a, int grid, cudaStream_t s) {
  if constexpr ((R0 * R1) % 16 == 0) {
    if (a.logP == 3) return launch_s3<R0, R1, 8, LOADM, STOREM>(a, grid, s);
  }
  if constexpr ((R0 * R1) % 32 == 0) {
    if (a.logP == 4) return launch_s3<R0, R1, 16, LOADM, STOREM>(a, grid, s);
  }
  return cudaErrorNotSupported;
}

// Two-stage plans for the contiguous passes; cudaErrorNotSupported when N or P has none.
template <int LOADM, int STOREM>
static cudaError_t launch_contig_fast(const DhtArgs<float> &a, int grid, cudaStream_t s) {
  switch (a.sp.N) {
    case 16: return launch_s3_p<4, 4, LOADM, STOREM>(a, grid, s);
    case 32: return launch_s3_p<8, 4, LOADM, STOREM>(a, grid, s);
    case 48: return launch_s3_p<16, 3, LOADM, STOREM>(a, grid, s);
    case 64: return launch_s3_p<8, 8, LOADM, STOREM>(a, grid, s);
    case 96: return launch_s3_p<16, 6, LOADM, STOREM>(a, grid, s);
    case 128: return launch_s3_p<16, 8, LOADM, STOREM>(a, grid, s);
    case 256: return launch_s3_p<16, 16, LOADM, STOREM>(a, grid, s);
    case 512: return launch_s3_p<32, 16, LOADM, STOREM>(a, grid, s);
    default: return cudaErrorNotSupported;
  }
}

// FP32 passes through the two-stage tiles where N and P allow; FP64 (ALU-bound,
// where the two-stage tiles measured slower) always takes the generic tile.
template <typename T>
static cudaError_t launch_fast(int pass, const DhtArgs<T> &a, int grid, cudaStream_t s) {
  if constexpr (sizeof(T) != 4) {
    return cudaErrorNotSupported;
  } else {
    switch (pass) {
      case PASS_A_RESID: return launch_contig_fast<LD_RESID, SO_PLAIN>(a, grid, s);
      case PASS_A_PLAIN: return launch_contig_fast<LD_PLAIN, SO_PLAIN>(a, grid, s);
      case PASS_E_PCG: return launch_contig_fast<LD_PLAIN, SO_PCG>(a, grid, s);
      case PASS_E_PLAIN: return launch_contig_fast<LD_PLAIN, SO_PLAIN>(a, grid, s);
      case PASS_B:
      case PASS_D: return launch_strided_fast<2, false>(a, grid, s);
      case PASS_C: return launch_strided_fast<1, true>(a, grid, s);
      default: return cudaErrorNotSupported;
    }
  }
}

static int g_pencils_override[kMaxN + 1] = {0};  // FP32 passes, per N (0 = default)
static int g_pencils_e_override[kMaxN + 1] = {0};  // FP32 pass E with the PCG update, per N (0 = as above)
static int g_strided_fast = 1;                    // two-stage strided passes where N allows
static int g_use_gtab = 1;                        // pass C reads the multiplier table where there is one

int set_use_gtab(int on) {
  if (on < 0 || on > 1) return 1;
  g_use_gtab = on;
  return 0;
}
int use_gtab() { return g_use_gtab; }

int set_strided_fast(int on) {
  if (on < 0 || on > 2) return 1;
  g_strided_fast = on;
  return 0;
}

int set_dht_pencils_override(int N, int P) {
  if (N < 8 || N > kMaxN) return 1;
  if (P != 0 && (P < 1 || (P & (P - 1)) || N % (2 * P) != 0 || dht_smem_bytes_t<float>(N, P, kMaxRank) > 200 * 1024))
    return 1;
  g_pencils_override[N] = P;
  return 0;
}

int set_dht_pencils_e_override(int N, int P) {
  if (N < 8 || N > kMaxN) return 1;
  if (P != 0 && (P < 1 || (P & (P - 1)) || N % (2 * P) != 0 || dht_smem_bytes_t<float>(N, P, 0) > 200 * 1024))
    return 1;
  g_pencils_e_override[N] = P;
  return 0;
}

int dht_tile_pencils(int N, int elem_bytes) {
  if (elem_bytes == 4 && N >= 8 && N <= kMaxN && g_pencils_override[N]) return g_pencils_override[N];
  // 2P real pencils per tile: 128-byte row segments where N allows, and two
  // ping-pong buffers of N (P+1) complex values within about 80 KB.
  int P = 128 / (2 * elem_bytes);
  while (P > 1 && ((N % (2 * P)) != 0 || 2L * N * (P + 1) * 2 * elem_bytes > 90 * 1024)) P >>= 1;
  return P;
}

template <typename T, int AXIS, int LOADM, int STOREM, bool SCALE, int XF = XF_HARTLEY>
static cudaError_t launch_one(const DhtArgs<T> &a, int grid, size_t smem, cudaStream_t s) {
  auto kern = k_dht<T, AXIS, LOADM, STOREM, SCALE, XF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dht_pass(int pass, const SpectralDev &sp, const T *in, T *out, T *r, const T *q, T *p, T *x,
                            RedBuf rb, bool first, bool check_done, cudaStream_t s) {
  const int N = sp.N;
  // pass E with the PCG update has a tile width of its own (its bulk-copy
  // staging of p and x adds 16 P N bytes of shared memory per block)
  const int Pe = (sizeof(T) == 4 && pass == PASS_E_PCG) ? g_pencils_e_override[N] : 0;
  int P = Pe ? Pe : dht_tile_pencils(N, (int)sizeof(T));
  // FP64 passes take tiles of at most 4 complex pencils: half the shared
  // memory, twice the blocks per SM to keep the FP64 pipe fed (at N = 256
  // the passes other than C went 3166 -> 3113 us per iteration; 2 pencils
  // are slower than 4). Pass C on the complex x2 route, 2 pencils per row:
  // 837.9 -> 827.6 us.
  if (sizeof(T) == 8 && P > 4) P = 4;
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
  a.stage = 0;
  a.ntiles = (int)(((long long)N * N) / (2 * P));
  if (!g_use_gtab) a.sp.gtab = nullptr;
  const int grid = a.ntiles < 8192 ? a.ntiles : 8192;
  const size_t smem = dht_smem_bytes_t<T>(N, P, pass == PASS_C ? sp.rank : 0);
  if (g_strided_fast) {
    const cudaError_t e = launch_fast<T>(pass, a, grid, s);
    if (e != cudaErrorNotSupported) return e;
  }
  // FP64: passes B, C, D take the complex x2 route (no Hartley combine in B
  // and D; pass C pairs the mirror rows). Every valid N gives pass C at least
  // 2 pencils, which its two halves need.
  if constexpr (sizeof(T) == 8) {
    if (dht_tile_pencils(N, 8) >= 2) {
      switch (pass) {
        case PASS_B: return launch_one<T, 2, LD_PLAIN, SO_PLAIN, false, XF_FWD>(a, grid, smem, s);
        case PASS_C: return launch_one<T, 1, LD_PLAIN, SO_PLAIN, true, XF_MIRROR>(a, grid, smem, s);
        case PASS_D: return launch_one<T, 2, LD_PLAIN, SO_PLAIN, false, XF_INV>(a, grid, smem, s);
        default: break;
      }
    }
  }
  switch (pass) {
    case PASS_A_RESID: return launch_one<T, 3, LD_RESID, SO_PLAIN, false>(a, grid, smem, s);
    case PASS_A_PLAIN: return launch_one<T, 3, LD_PLAIN, SO_PLAIN, false>(a, grid, smem, s);
    case PASS_B:
    case PASS_D: return launch_one<T, 2, LD_PLAIN, SO_PLAIN, false>(a, grid, smem, s);
    case PASS_C: return launch_one<T, 1, LD_PLAIN, SO_PLAIN, true>(a, grid, smem, s);
    case PASS_E_PCG: return launch_one<T, 3, LD_PLAIN, SO_PCG, false>(a, grid, smem, s);
    case PASS_E_PLAIN: return launch_one<T, 3, LD_PLAIN, SO_PLAIN, false>(a, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

// 2D passes on an N x N field (x2 contiguous): the same tiles with N rows in
// place of N^2. PASS_A_* / PASS_E_*: row transforms (the x3 tile); PASS_C: the
// column transform (the x2 tile of the single line 0), scaled by G(k, 0, k2)
// = G2(k, k2) and transformed again. Scale and factors are set up for 2D.
template <typename T>
cudaError_t launch_dht_pass_2d(int pass, const SpectralDev &sp, const T *in, T *out, T *r, const T *q, T *p, T *x,
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
  a.stage = 0;
  a.ntiles = N / (2 * P);
  const int grid = a.ntiles;
  const size_t smem = dht_smem_bytes_t<T>(N, P, pass == PASS_C ? sp.rank : 0);
  switch (pass) {
    case PASS_A_RESID: return launch_one<T, 3, LD_RESID, SO_PLAIN, false>(a, grid, smem, s);
    case PASS_A_PLAIN: return launch_one<T, 3, LD_PLAIN, SO_PLAIN, false>(a, grid, smem, s);
    case PASS_C: return launch_one<T, 2, LD_PLAIN, SO_PLAIN, true>(a, grid, smem, s);
    case PASS_E_PCG: return launch_one<T, 3, LD_PLAIN, SO_PCG, false>(a, grid, smem, s);
    case PASS_E_PLAIN: return launch_one<T, 3, LD_PLAIN, SO_PLAIN, false>(a, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_dht_pass_2d<double>(int, const SpectralDev &, const double *, double *, double *,
                                                const double *, double *, double *, RedBuf, bool, bool,
                                                cudaStream_t);

template cudaError_t launch_dht_pass<double>(int, const SpectralDev &, const double *, double *, double *,
                                             const double *, double *, double *, RedBuf, bool, bool, cudaStream_t);
template cudaError_t launch_dht_pass<float>(int, const SpectralDev &, const float *, float *, float *, const float *,
                                            float *, float *, RedBuf, bool, bool, cudaStream_t);

}  // namespace sq
