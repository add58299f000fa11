// Host side of libsq: handles, preconditioner tables, the PCG driver and the
// C ABI declared in include/sq.h.
//
// PCG (Sec. 4.1, Eqs. 24-25; Hestenes-Stiefel form of Matlab's pcg) with the
// iteration split into six kernels; all scalars stay on the device:
//   K  q = A p                 ; p.q      -> alpha = rz/pq
//   A  x3 Hartley pass of r -= alpha q    ; ||r||^2 -> iter++, stop test
//   B  x2 pass
//   C  x1 pass, G scaling, x1 pass        ; r.z    -> beta
//   D  x2 pass
//   E  x3 pass -> z; x += alpha p; p = z + beta p
// Once the stop test fires every later kernel returns at entry; the host only
// polls a pinned copy of the `done` flag one chunk of iterations behind, so the
// GPU queue never drains while the host waits.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "common.cuh"

using namespace sq;

struct sq_coeffs {
  int L, n, N;
  double a_lo, a_hi;
  int sub_lo = 0, sub_hi = 1 << 30;  // inclusion cube of every cell (default: the whole cell)
  int levels = 2;                    // K: phase byte v reads level min(v, K - 1)
  double a_up[kMaxLevels - 2] = {0.0, 0.0};  // values of levels 2 .. K-1
  uint8_t *d_phase;
  cudaStream_t stream;
  Scalars *d_st;       // reduction scalars for operator / A_hom calls
  double *d_partials;  // kMaxQ * kMaxPartials
  Scalars *h_st;       // pinned
};

struct sq_precond {
  int N, rank;
  std::vector<double> t, w;  // exponential-sum nodes and weights (empty for other factors)
  std::vector<double> f;     // host factors, 3 x rank x N (unscaled; see precond_create)
  SpectralDev sp64, sp32;
  void *d_mem;
};

struct sq_workspace {
  int N, precision;
  double *f64;   // r, p, q, Y (SQ_FP64)
  float *f32;    // r, p, q, Y, d (SQ_FP32_REFINE)
  Scalars *d_st;  // [0] outer / FP64 solve, [1] inner FP32 solve
  double *d_partials;
  Scalars *h_st;  // pinned copies of the two scalar blocks
  int *h_poll;    // pinned, 2 slots
  cudaEvent_t ev[2];
  // CUDA graphs of kPollChunk steady-state PCG iterations (see pcg_loop),
  // each with the signature of the launch parameters it bakes in
  struct IterGraph {
    std::vector<uint64_t> sig;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int kernels;
  };
  std::vector<IterGraph> graphs;
};

namespace {

#define SQ_CK(call)                                   \
  do {                                                \
    cudaError_t _e = (call);                          \
    if (_e != cudaSuccess) return SQ_ECUDA;           \
  } while (0)

// ---------------------------------------------------------------- profiling
// Optional CUDA-event pairs around every kernel launch, summed per class.
enum ProfClass : int {
  PC_COEFF = 0, PC_MATVEC, PC_RESID, PC_DHT_A, PC_DHT_B, PC_DHT_C, PC_DHT_E, PC_VECTOR, PC_AHOM, PC_SCALAR,
  PC_BATCH_INNER, PC_BATCH_LOOP, PC_COUNT
};
const char *const kProfNames[PC_COUNT] = {"coeff_gen",  "stencil_matvec", "stencil_resid_rhs", "dht_x3_in",
                                          "dht_x2",     "dht_x1_scale",   "dht_x3_out",        "vector",
                                          "ahom",       "scalars",        "batch_inner",
                                          "batch_inner_loop"};
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> cls;
  size_t used = 0;
};
Prof g_prof;
double g_prof_work_ms[PC_COUNT] = {0};  // of the last sq_profile_read
int64_t g_prof_work_n[PC_COUNT] = {0};

const size_t kNoProf = (size_t)-1;

int64_t g_launches = 0;  // every kernel launch through SQ_LAUNCH since the library was loaded

size_t prof_begin(int cls, cudaStream_t s) {
  ++g_launches;
  if (!g_prof.on) return kNoProf;
  while (g_prof.pool.size() < g_prof.used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return kNoProf;
    g_prof.pool.push_back(e);
  }
  const size_t i = g_prof.used;
  if (cudaEventRecord(g_prof.pool[i], s) != cudaSuccess) return kNoProf;
  g_prof.cls.push_back(cls);
  g_prof.used += 2;
  return i;
}

void prof_end(size_t i, cudaStream_t s) {
  if (i != kNoProf) cudaEventRecord(g_prof.pool[i + 1], s);
}

#define SQ_LAUNCH(cls, s, call)                      \
  do {                                               \
    const size_t _pi = prof_begin((cls), (s));       \
    cudaError_t _e = (call);                         \
    prof_end(_pi, (s));                              \
    if (_e != cudaSuccess) return SQ_ECUDA;          \
  } while (0)

bool valid_N(int N) {
  if (N < 8 || N > kMaxN || (N & 1)) return false;
  int m = N;
  while (m % 2 == 0) m /= 2;
  if (m % 3 == 0) m /= 3;
  return m == 1;
}

CellsDev cells_dev(const sq_coeffs *c) {
  CellsDev d;
  d.phase = c->d_phase;
  d.L = c->L;
  d.n = c->n;
  d.N = c->N;
  d.a_lo = c->a_lo;
  d.a_hi = c->a_hi;
  d.sub_lo = c->sub_lo;
  d.sub_hi = c->sub_hi;
  d.layers = c->levels - 1;
  for (int l = 0; l < kMaxLevels - 2; ++l) d.a_up[l] = c->a_up[l];
  fill_tables(d);
  return d;
}

int alloc_coeffs(int L, int n, double a_lo, double a_hi, cudaStream_t s, sq_coeffs **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (L < 1 || n < 2 || !valid_N(L * n)) return SQ_EINVAL;
  if (!(a_lo > 0.0) || !(a_hi > 0.0) || !std::isfinite(a_lo) || !std::isfinite(a_hi)) return SQ_EINVAL;
  sq_coeffs *c = new (std::nothrow) sq_coeffs();
  if (!c) return SQ_ENOMEM;
  c->L = L;
  c->n = n;
  c->N = L * n;
  c->a_lo = a_lo;
  c->a_hi = a_hi;
  c->stream = s;
  if (cudaMalloc(&c->d_phase, (size_t)L * L * L) != cudaSuccess ||
      cudaMalloc(&c->d_st, sizeof(Scalars)) != cudaSuccess ||
      cudaMalloc(&c->d_partials, sizeof(double) * kMaxQ * kMaxPartials) != cudaSuccess ||
      cudaMallocHost(&c->h_st, sizeof(Scalars)) != cudaSuccess) {
    sq_coeffs_destroy(c);
    return SQ_ENOMEM;
  }
  if (cudaMemsetAsync(c->d_st, 0, sizeof(Scalars), s) != cudaSuccess) {
    sq_coeffs_destroy(c);
    return SQ_ECUDA;
  }
  *out = c;
  return SQ_OK;
}

// radix plan: 3 (if present) last, powers of two as 8s then one 4 or 2
int radix_plan(int N, int *rad) {
  int m = N, ns = 0, t = 0;
  while (m % 3 == 0) {
    m /= 3;
    ++t;
  }
  int e = 0;
  while (m > 1) {
    m /= 2;
    ++e;
  }
  if (e == 4) {
    rad[ns++] = 4;
    rad[ns++] = 4;
    e = 0;
  }
  while (e >= 3) {
    rad[ns++] = 8;
    e -= 3;
  }
  if (e == 2) rad[ns++] = 4;
  if (e == 1) rad[ns++] = 2;
  for (int i = 0; i < t; ++i) rad[ns++] = 3;
  return ns;
}

// Rank-R exponential sum for 1/x on [lambda_min, 12] (Sec. 4.2, Eq. 34 read as
// the trapezoid rule for 1/x = int exp(s - x e^s) ds): three error terms --
// lower truncation 12 e^{s_lo}, upper truncation exp(-lambda_min e^{s_hi}) and
// the step error exp(-pi^2/eta) -- are balanced at one level eps, found by
// bisection on ln(eps); nodes s_r = s_lo + r eta, t_r = e^{s_r}, w_r = eta e^{s_r}.
// dim = 2 or 3: the spectrum lies in [lambda_min, 4 dim].
void sinc_nodes(int N, int R, std::vector<double> &t, std::vector<double> &w, int dim = 3) {
  const double pi = 3.14159265358979323846;
  const double sn = std::sin(pi / N);
  const double lam_min = 4.0 * sn * sn;
  const double xmax = 4.0 * dim;
  double lo = std::log(1e-300), hi = std::log(0.5);
  auto eta_of = [&](double le, double *slo) {
    const double s_lo = le - std::log(xmax);
    const double s_hi = std::log(-le / lam_min);
    *slo = s_lo;
    return (s_hi - s_lo) / (R - 1);
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    double slo;
    const double eta = eta_of(mid, &slo);
    if (std::exp(-pi * pi / eta) > std::exp(mid))
      lo = mid;
    else
      hi = mid;
  }
  double s_lo;
  const double eta = eta_of(0.5 * (lo + hi), &s_lo);
  t.resize(R);
  w.resize(R);
  for (int r = 0; r < R; ++r) {
    const double s = s_lo + eta * r;
    t[r] = std::exp(s);
    w[r] = eta * std::exp(s);
  }
}

// Least-squares solve min ||E w - 1|| (M x R, column-major copy) by Householder QR.
// Fails (returns false) when the fit is numerically singular: the ratio of the
// largest to the smallest |diagonal entry| of the triangular factor above 1e10
// (exponential fits over a narrow spectrum with many terms), where the weights
// would be rounding noise.
bool lsq_ones(std::vector<double> E, int M, int R, std::vector<double> &w) {
  if (R < 1 || M < 2 * R) return false;  // too few distinct spectral values for a fit
  std::vector<double> rhs(M, 1.0);
  for (int k = 0; k < R; ++k) {
    double nrm = 0.0;
    for (int i = k; i < M; ++i) nrm += E[(size_t)k * M + i] * E[(size_t)k * M + i];
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) return false;
    const double a0 = E[(size_t)k * M + k];
    const double alpha = (a0 > 0) ? -nrm : nrm;
    std::vector<double> v(E.begin() + (size_t)k * M + k, E.begin() + (size_t)k * M + M);
    v[0] -= alpha;
    double vv = 0.0;
    for (double x : v) vv += x * x;
    if (!(vv > 0.0)) return false;
    for (int j = k; j < R; ++j) {
      double d = 0.0;
      for (int i = k; i < M; ++i) d += v[i - k] * E[(size_t)j * M + i];
      d = 2.0 * d / vv;
      for (int i = k; i < M; ++i) E[(size_t)j * M + i] -= d * v[i - k];
    }
    double d = 0.0;
    for (int i = k; i < M; ++i) d += v[i - k] * rhs[i];
    d = 2.0 * d / vv;
    for (int i = k; i < M; ++i) rhs[i] -= d * v[i - k];
  }
  double dmax = 0.0, dmin = std::numeric_limits<double>::infinity();
  for (int k = 0; k < R; ++k) {
    const double d = std::fabs(E[(size_t)k * M + k]);
    dmax = std::max(dmax, d);
    dmin = std::min(dmin, d);
  }
  if (!(dmin > 0.0) || dmax > 1e10 * dmin) return false;
  w.assign(R, 0.0);
  for (int k = R - 1; k >= 0; --k) {
    double s = rhs[k];
    for (int j = k + 1; j < R; ++j) s -= E[(size_t)j * M + k] * w[j];
    const double d = E[(size_t)k * M + k];
    if (!(std::fabs(d) > 0.0)) return false;
    w[k] = s / d;
  }
  return true;
}

// Largest relative error |x G(x) - 1| of the exponential sum over the values xs.
double exp_sum_error(const std::vector<double> &xs, const std::vector<double> &t, const std::vector<double> &w) {
  double err = 0.0;
  for (double x : xs) {
    double g = 0.0;
    for (size_t r = 0; r < t.size(); ++r) g += w[r] * std::exp(-t[r] * x);
    err = std::max(err, std::fabs(x * g - 1.0));
  }
  return err;
}

// Rank-R factors used by the library: geometric nodes t_r between e^a and e^b,
// weights w_r by least squares on the relative error x G_R(x) - 1 over a
// log-uniform sample of the discrete spectrum {l_i + l_j + l_k > 0} (dim 3;
// {l_i + l_j > 0} for dim 2); (a, b) is chosen on a grid to minimise the
// largest sampled error with all w_r > 0 among the fits that are not
// numerically singular (see lsq_ones). The result is kept only if its
// largest error over the whole spectrum is below that of the balanced
// trapezoid rule (which is used otherwise, and for R > 32).
void rank_r_nodes(int N, int R, std::vector<double> &t, std::vector<double> &w, int dim = 3) {
  sinc_nodes(N, R, t, w, dim);
  if (R > 32) return;
  const double pi = 3.14159265358979323846;
  const int H = N / 2;
  std::vector<double> lam(H + 1);
  for (int k = 0; k <= H; ++k) {
    const double sn = std::sin(pi * k / N);
    lam[k] = 4.0 * sn * sn;
  }
  std::vector<double> xs;
  if (dim == 2) {
    xs.reserve((size_t)(H + 1) * (H + 2) / 2);
    for (int i = 0; i <= H; ++i)
      for (int j = i; j <= H; ++j)
        if (lam[i] + lam[j] > 0.0) xs.push_back(lam[i] + lam[j]);
  } else {
    xs.reserve((size_t)(H + 1) * (H + 2) * (H + 3) / 6);
    for (int i = 0; i <= H; ++i)
      for (int j = i; j <= H; ++j)
        for (int k = j; k <= H; ++k) {
          const double g = lam[i] + lam[j] + lam[k];
          if (g > 0.0) xs.push_back(g);
        }
  }
  std::sort(xs.begin(), xs.end());
  std::vector<double> u;  // distinct spectral values
  for (double x : xs)
    if (u.empty() || x > u.back() * (1.0 + 1e-12)) u.push_back(x);
  // log-uniform sample: the distinct value nearest to each point of a geometric grid
  std::vector<double> smp;
  const int K = 3000;
  const double x0 = u.front(), x1 = u.back();
  for (int m = 0; m < K; ++m) {
    const double xt = x0 * std::pow(x1 / x0, (double)m / (K - 1));
    auto it = std::lower_bound(u.begin(), u.end(), xt);
    double pick = (it == u.end()) ? u.back() : *it;
    if (it != u.begin() && (it == u.end() || std::fabs(*(it - 1) - xt) < std::fabs(pick - xt))) pick = *(it - 1);
    if (smp.empty() || pick > smp.back()) smp.push_back(pick);
  }
  const int M = (int)smp.size();
  if (M < 2 * R) return;
  const double lam_min = lam[1];
  const int ng = (R <= 16) ? 40 : 20;
  double best = std::numeric_limits<double>::infinity();
  std::vector<double> bt, bw, tt(R), ww, E((size_t)M * R);
  for (int ia = 0; ia < ng; ++ia) {
    const double a = -std::log(4.0 * dim) - 6.0 + 7.0 * ia / (ng - 1);
    for (int ib = 0; ib < ng; ++ib) {
      const double b = std::log(1.0 / lam_min) - 1.0 + 5.0 * ib / (ng - 1);
      for (int r = 0; r < R; ++r) tt[r] = std::exp(a + (b - a) * r / (R - 1));
      for (int r = 0; r < R; ++r)
        for (int i = 0; i < M; ++i) E[(size_t)r * M + i] = smp[i] * std::exp(-tt[r] * smp[i]);
      if (!lsq_ones(E, M, R, ww)) continue;
      bool pos = true;
      for (double x : ww) pos = pos && (x > 0.0);
      if (!pos) continue;
      double err = 0.0;
      for (int i = 0; i < M; ++i) {
        double gsum = 0.0;
        for (int r = 0; r < R; ++r) gsum += ww[r] * E[(size_t)r * M + i];
        err = std::max(err, std::fabs(gsum - 1.0));
      }
      if (err < best) {
        best = err;
        bt = tt;
        bw = ww;
      }
    }
  }
  if (!bt.empty() && exp_sum_error(u, bt, bw) < exp_sum_error(u, t, w)) {
    t = bt;
    w = bw;
  }
}

template <typename T>
RedBuf redbuf(Scalars *st, double *partials) {
  RedBuf rb;
  rb.st = st;
  rb.partials = partials;
  return rb;
}

__global__ void k_scalars_reset(Scalars *st, double tolrel2, int max_iter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    Scalars z;
    memset(&z, 0, sizeof(z));
    z.tolrel2 = tolrel2;
    z.max_iter = max_iter;
    *st = z;
  }
}

// Inner FP32 solve of A d = r (r = FP32 copy of the outer residual): its
// ||b||^2 is the outer residual norm.
__global__ void k_inner_init(Scalars *in, const Scalars *outer, double tolrel2, int max_iter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    Scalars z;
    memset(&z, 0, sizeof(z));
    z.tolrel2 = tolrel2;
    z.max_iter = max_iter;
    z.bb = outer->rr_true;
    z.tol2 = tolrel2 * outer->rr_true;
    z.done = (outer->rr_true > 0.0) ? 0 : 1;
    *in = z;
  }
}

template <typename T>
const SpectralDev &spec(const sq_precond *pc);
template <>
const SpectralDev &spec<double>(const sq_precond *pc) { return pc->sp64; }
template <>
const SpectralDev &spec<float>(const sq_precond *pc) { return pc->sp32; }

// Preconditioned residual from r: z passes with p = z (first) inside PCG.
template <typename T>
int precond_first(const sq_precond *pc, T *r, T *Y, T *p, RedBuf rb, cudaStream_t s) {
  const SpectralDev &sp = spec<T>(pc);
  SQ_LAUNCH(PC_DHT_A, s, launch_dht_pass<T>(PASS_A_PLAIN, sp, r, Y, nullptr, nullptr, nullptr, nullptr, rb, true, true, s));
  SQ_LAUNCH(PC_DHT_B, s, launch_dht_pass<T>(PASS_B, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, true, true, s));
  SQ_LAUNCH(PC_DHT_C, s, launch_dht_pass<T>(PASS_C, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, true, true, s));
  SQ_LAUNCH(PC_DHT_B, s, launch_dht_pass<T>(PASS_D, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, true, true, s));
  SQ_LAUNCH(PC_DHT_E, s, launch_dht_pass<T>(PASS_E_PCG, sp, Y, nullptr, nullptr, nullptr, p, nullptr, rb, true, true, s));
  return SQ_OK;
}

template <typename T>
int pcg_iteration(const sq_coeffs *c, const sq_precond *pc, T *x, T *r, T *p, T *q, T *Y, RedBuf rb,
                  cudaStream_t s) {
  const SpectralDev &sp = spec<T>(pc);
  const CellsDev cd = cells_dev(c);
  SQ_LAUNCH(PC_MATVEC, s, (launch_stencil<T, T>(cd, ST_MATVEC, 0, p, q, rb, FIN_ALPHA, true, s)));
  SQ_LAUNCH(PC_DHT_A, s, launch_dht_pass<T>(PASS_A_RESID, sp, r, Y, r, q, nullptr, nullptr, rb, false, true, s));
  SQ_LAUNCH(PC_DHT_B, s, launch_dht_pass<T>(PASS_B, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, false, true, s));
  SQ_LAUNCH(PC_DHT_C, s, launch_dht_pass<T>(PASS_C, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, false, true, s));
  SQ_LAUNCH(PC_DHT_B, s, launch_dht_pass<T>(PASS_D, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, false, true, s));
  SQ_LAUNCH(PC_DHT_E, s, launch_dht_pass<T>(PASS_E_PCG, sp, Y, nullptr, nullptr, nullptr, p, x, rb, false, true, s));
  return SQ_OK;
}

// ------------------------------------------------------- iteration graphs
// Single solves replay a CUDA graph of kPollChunk steady-state iterations
// (six kernels each) instead of launching every kernel from the host: at
// small N the host's launch rate, not the GPU, paced a solve. A graph bakes in
// every launch parameter, so it is found by a signature of them: the field
// pointers, the reduction buffers, the coefficient and spectral descriptors
// (field by field) and the option epoch, which every option or tile change
// bumps. A workspace keeps the last kMaxGraphs graphs (one per output field
// and precision in typical use). Profiling launches directly (its events
// cannot sit inside a graph), and so does a call whose stream is being
// captured already.
int g_option_epoch = 0;  // bumped by sq_set_option and sq_set_tiles
int g_pcg_graphs = 1;    // SQ_OPT_PCG_GRAPHS
constexpr size_t kMaxGraphs = 8;
}  // namespace

namespace sq {
int pcg_graphs_enabled() { return g_pcg_graphs; }
int option_epoch() { return g_option_epoch; }
}  // namespace sq

namespace {

template <typename T>
std::vector<uint64_t> iter_signature(const sq_coeffs *c, const sq_precond *pc, const T *x, const T *r, const T *p,
                                     const T *q, const T *Y, RedBuf rb) {
  std::vector<uint64_t> v;
  auto add = [&](uint64_t u) { v.push_back(u); };
  auto addp = [&](const void *ptr) { add((uint64_t)(uintptr_t)ptr); };
  auto addd = [&](double d) {
    uint64_t u;
    memcpy(&u, &d, sizeof(u));
    add(u);
  };
  add(sizeof(T));
  add((uint64_t)g_option_epoch);
  addp(x), addp(r), addp(p), addp(q), addp(Y), addp(rb.st), addp(rb.partials);
  const CellsDev cd = cells_dev(c);
  addp(cd.phase), add(cd.L), add(cd.n), add(cd.N), addd(cd.a_lo), addd(cd.a_hi), add((uint64_t)cd.sub_lo);
  add((uint64_t)cd.sub_hi), add(cd.layers);
  for (double a : cd.a_up) addd(a);
  const SpectralDev &sp = spec<T>(pc);
  add(sp.N), add(sp.rank), addp(sp.tw), addp(sp.lam), addp(sp.u), addd(sp.scale), addp(sp.gtab);
  return v;
}

// The graph for these launch parameters: found in the workspace, or
// captured (on a private stream) and instantiated.
template <typename T>
int iter_graph(sq_workspace *w, const sq_coeffs *c, const sq_precond *pc, T *x, T *r, T *p, T *q, T *Y, RedBuf rb,
               cudaGraphExec_t *exec, int *kernels) {
  std::vector<uint64_t> sig = iter_signature<T>(c, pc, x, r, p, q, Y, rb);
  for (const sq_workspace::IterGraph &e : w->graphs) {
    if (e.sig == sig) {
      *exec = e.exec;
      *kernels = e.kernels;
      return SQ_OK;
    }
  }
  if (w->graphs.size() >= kMaxGraphs) {
    cudaGraphExecDestroy(w->graphs.front().exec);
    cudaGraphDestroy(w->graphs.front().graph);
    w->graphs.erase(w->graphs.begin());
  }
  cudaStream_t cs;
  SQ_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const int64_t l0 = g_launches;
  int st = SQ_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = SQ_ECUDA;
  for (int i = 0; st == SQ_OK && i < kPollChunk; ++i) st = pcg_iteration<T>(c, pc, x, r, p, q, Y, rb, cs);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g) st = SQ_ECUDA;
  cudaGraphExec_t ge = nullptr;
  if (st == SQ_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) st = SQ_ECUDA;
  cudaStreamDestroy(cs);
  const int nk = (int)(g_launches - l0);
  g_launches = l0;  // counted when replayed
  if (st != SQ_OK) {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    return st;
  }
  w->graphs.push_back(sq_workspace::IterGraph{std::move(sig), g, ge, nk});
  *exec = ge;
  *kernels = nk;
  return SQ_OK;
}

// Runs PCG iterations until the device sets `done` (converged, max_iter or
// breakdown) or `budget` iterations were launched. Polls one chunk behind.
template <typename T>
int pcg_loop(sq_workspace *w, const sq_coeffs *c, const sq_precond *pc, T *x, T *r, T *p, T *q, T *Y, RedBuf rb,
             int budget, cudaStream_t s) {
  // Iterations per poll: the host learns of convergence up to two chunks
  // late, and every iteration launched after it costs six launches that exit
  // at entry (about 10 us each for the FP32 passes at N = 256). Measured at
  // N = 256, FP32 rank 8: 49.2 / 51.5 / 52.4 solves/s for chunks of 8 / 4 / 2;
  // the queue stays ahead of the GPU at 2 (the host enqueues an iteration in
  // far less than the GPU runs it).
  const int chunk = kPollChunk;
  int launched = 0, slot = 0;
  bool pending[2] = {false, false};
  w->h_poll[0] = w->h_poll[1] = 0;
  const size_t done_off = offsetof(Scalars, done);
  cudaGraphExec_t gx = nullptr;
  int gk = 0;
  if (g_pcg_graphs && !g_prof.on && budget >= chunk) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    SQ_CK(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone && iter_graph<T>(w, c, pc, x, r, p, q, Y, rb, &gx, &gk) != SQ_OK) {
      gx = nullptr;  // no graph (capture or instantiation failed): launch one by one
      (void)cudaGetLastError();
    }
  }
  while (launched < budget) {
    const int nb = (budget - launched < chunk) ? budget - launched : chunk;
    if (gx && nb == chunk) {
      SQ_CK(cudaGraphLaunch(gx, s));
      g_launches += gk;
    } else {
      for (int i = 0; i < nb; ++i) {
        int st = pcg_iteration<T>(c, pc, x, r, p, q, Y, rb, s);
        if (st != SQ_OK) return st;
      }
    }
    launched += nb;
    SQ_CK(cudaMemcpyAsync(&w->h_poll[slot], reinterpret_cast<char *>(rb.st) + done_off, sizeof(int),
                          cudaMemcpyDeviceToHost, s));
    SQ_CK(cudaEventRecord(w->ev[slot], s));
    pending[slot] = true;
    const int other = slot ^ 1;
    if (pending[other]) {
      SQ_CK(cudaEventSynchronize(w->ev[other]));
      pending[other] = false;
      if (w->h_poll[other]) break;
    }
    slot = other;
  }
  return SQ_OK;
}

int read_scalars(Scalars *h, const Scalars *d, cudaStream_t s) {
  SQ_CK(cudaMemcpyAsync(h, d, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  SQ_CK(cudaStreamSynchronize(s));
  return SQ_OK;
}

int solve_fp64(const sq_coeffs *c, const sq_precond *pc, sq_workspace *w, int dir, double tol, int max_iter,
               const double *x0, double *psi, sq_solve_info *info, cudaStream_t s) {
  const long long n3 = (long long)c->N * c->N * c->N;
  double *r = w->f64, *p = r + n3, *q = p + n3, *Y = q + n3;
  const RedBuf rb = redbuf<double>(&w->d_st[0], w->d_partials);
  const CellsDev cd = cells_dev(c);
  SQ_LAUNCH(PC_SCALAR, s, (k_scalars_reset<<<1, 1, 0, s>>>(rb.st, tol * tol, max_iter), cudaGetLastError()));
  Scalars *h = &w->h_st[0];
  bool used_guess = false;
  if (x0) {
    if (x0 != psi) SQ_CK(cudaMemcpyAsync(psi, x0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s));
    SQ_LAUNCH(PC_RESID, s, (launch_stencil<double, double>(cd, ST_RESID, dir, psi, r, rb, FIN_RESID, false, s)));
    // the residual decides on the guess: keep it only if ||b - A x0|| < ||b||
    int st = read_scalars(h, rb.st, s);
    if (st != SQ_OK) return st;
    used_guess = h->rr < h->bb;
  }
  if (!used_guess) {
    SQ_CK(cudaMemsetAsync(psi, 0, sizeof(double) * n3, s));
    SQ_LAUNCH(PC_RESID, s, (launch_stencil<double, double>(cd, ST_RHS, dir, nullptr, r, rb, FIN_RESID, false, s)));
  }
  for (int restart = 0; restart < 4; ++restart) {
    int st = precond_first<double>(pc, r, Y, p, rb, s);
    if (st != SQ_OK) return st;
    st = pcg_loop<double>(w, c, pc, psi, r, p, q, Y, rb, max_iter, s);
    if (st != SQ_OK) return st;
    SQ_LAUNCH(PC_VECTOR, s, launch_x_final_sum<double>(psi, p, rb, n3, s));
    SQ_LAUNCH(PC_VECTOR, s, launch_sub_mean<double>(psi, rb, n3, s));
    SQ_LAUNCH(PC_RESID, s, (launch_stencil<double, double>(cd, ST_RESID, dir, psi, r, rb, FIN_RESID, false, s)));
    st = read_scalars(h, rb.st, s);
    if (st != SQ_OK) return st;
    if (h->done || h->iter >= max_iter || h->breakdown) break;
  }
  if (info) {
    info->iters = h->iter;
    info->outer_steps = 1;
    info->used_guess = used_guess ? 1 : 0;
    info->relres = (h->bb > 0.0) ? std::sqrt(h->rr / h->bb) : 0.0;
    info->relres_true = (h->bb > 0.0) ? std::sqrt(h->rr_true / h->bb) : 0.0;
    info->status = (h->bb == 0.0 || info->relres_true <= tol) ? SQ_OK : SQ_ENOCONV;
  }
  const bool ok = (h->bb == 0.0) || std::sqrt(h->rr_true / h->bb) <= tol;
  return ok ? SQ_OK : SQ_ENOCONV;
}

int solve_fp32_refine(const sq_coeffs *c, const sq_precond *pc, sq_workspace *w, int dir, double tol,
                      int max_iter, const double *x0, double *psi, sq_solve_info *info, cudaStream_t s) {
  const long long n3 = (long long)c->N * c->N * c->N;
  float *r = w->f32, *p = r + n3, *q = p + n3, *Y = q + n3, *d = Y + n3;
  const RedBuf ro = redbuf<double>(&w->d_st[0], w->d_partials);
  const RedBuf ri = redbuf<double>(&w->d_st[1], w->d_partials);
  const CellsDev cd = cells_dev(c);
  const double tol_in = inner_tol();
  SQ_LAUNCH(PC_SCALAR, s, (k_scalars_reset<<<1, 1, 0, s>>>(ro.st, tol * tol, max_iter), cudaGetLastError()));
  Scalars *ho = &w->h_st[0], *hi = &w->h_st[1];
  bool used_guess = false;
  if (x0) {
    if (x0 != psi) SQ_CK(cudaMemcpyAsync(psi, x0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s));
    SQ_LAUNCH(PC_RESID, s, (launch_stencil<double, float>(cd, ST_RESID, dir, psi, r, ro, FIN_RESID, false, s)));
    int st = read_scalars(ho, ro.st, s);
    if (st != SQ_OK) return st;
    used_guess = ho->rr_true < ho->bb;  // keep the guess only if it reduces the residual
  }
  if (!used_guess) SQ_CK(cudaMemsetAsync(psi, 0, sizeof(double) * n3, s));
  int total_inner = 0, outer = 0;
  double relres_in = 0.0;
  bool timed_out = false;
  for (;;) {
    // FP64 true residual, stored as the FP32 right-hand side of the correction
    // (from psi = 0 it is b itself: the right-hand-side sweep, no operator)
    if (outer == 0 && !used_guess)
      SQ_LAUNCH(PC_RESID, s, (launch_stencil<double, float>(cd, ST_RHS, dir, nullptr, r, ro, FIN_RESID, false, s)));
    else
      SQ_LAUNCH(PC_RESID, s, (launch_stencil<double, float>(cd, ST_RESID, dir, psi, r, ro, FIN_RESID, false, s)));
    int st = read_scalars(ho, ro.st, s);
    if (st != SQ_OK) return st;
    if (ho->done || total_inner >= max_iter || outer >= 30) break;
    const int budget = max_iter - total_inner;
    // each inner solve cuts its residual by tol_in, or just enough for the
    // outer tolerance when that is less (the last step)
    const double need = 0.9 * tol * std::sqrt(ho->bb / ho->rr_true);
    const double tin = std::max(tol_in, need);
    SQ_LAUNCH(PC_SCALAR, s, (k_inner_init<<<1, 1, 0, s>>>(ri.st, ro.st, tin * tin, budget), cudaGetLastError()));
    SQ_CK(cudaMemsetAsync(d, 0, sizeof(float) * n3, s));
    st = precond_first<float>(pc, r, Y, p, ri, s);
    if (st != SQ_OK) return st;
    st = pcg_loop<float>(w, c, pc, d, r, p, q, Y, ri, budget, s);
    if (st != SQ_OK) return st;
    SQ_LAUNCH(PC_VECTOR, s, launch_x_final_sum<float>(d, p, ri, n3, s));
    SQ_LAUNCH(PC_VECTOR, s, launch_add_f32_to_f64(psi, d, n3, s));
    st = read_scalars(hi, ri.st, s);
    if (st != SQ_OK) return st;
    // a bounded staging wait gave up: the kernel read its operands from
    // global memory instead, so the step is complete; the solve carries on
    // and reports SQ_ETIMEOUT at the end
    timed_out = timed_out || hi->fault;
    relres_in = (hi->bb > 0.0) ? std::sqrt(hi->rr / hi->bb) : 0.0;
    total_inner += hi->iter;
    ++outer;
    if (hi->iter == 0 && !hi->conv) break;  // no progress possible
  }
  SQ_LAUNCH(PC_VECTOR, s, launch_x_final_sum<double>(psi, nullptr, ro, n3, s));  // x_pending = 0 after FIN_RESID
  SQ_LAUNCH(PC_VECTOR, s, launch_sub_mean<double>(psi, ro, n3, s));
  SQ_CK(cudaStreamSynchronize(s));
  const double rel = (ho->bb > 0.0) ? std::sqrt(ho->rr_true / ho->bb) : 0.0;
  const int status = timed_out ? SQ_ETIMEOUT : (ho->bb == 0.0 || rel <= tol) ? SQ_OK : SQ_ENOCONV;
  if (info) {
    info->iters = total_inner;
    info->outer_steps = outer;
    info->used_guess = used_guess ? 1 : 0;
    info->relres = relres_in;
    info->relres_true = rel;
    info->status = status;
  }
  return status;
}

template <typename T>
int apply_precond_t(const sq_precond *pc, sq_workspace *w, const T *r, T *z, T *Y, cudaStream_t s) {
  const SpectralDev &sp = spec<T>(pc);
  const RedBuf rb = redbuf<double>(&w->d_st[0], w->d_partials);
  SQ_LAUNCH(PC_SCALAR, s, (k_scalars_reset<<<1, 1, 0, s>>>(rb.st, 0.0, 1), cudaGetLastError()));
  SQ_LAUNCH(PC_DHT_A, s, launch_dht_pass<T>(PASS_A_PLAIN, sp, r, Y, nullptr, nullptr, nullptr, nullptr, rb, true, false, s));
  SQ_LAUNCH(PC_DHT_B, s, launch_dht_pass<T>(PASS_B, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, true, false, s));
  SQ_LAUNCH(PC_DHT_C, s, launch_dht_pass<T>(PASS_C, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, true, false, s));
  SQ_LAUNCH(PC_DHT_B, s, launch_dht_pass<T>(PASS_D, sp, Y, Y, nullptr, nullptr, nullptr, nullptr, rb, true, false, s));
  SQ_LAUNCH(PC_DHT_E, s, launch_dht_pass<T>(PASS_E_PLAIN, sp, Y, z, nullptr, nullptr, nullptr, nullptr, rb, true, false, s));
  return SQ_OK;
}

}  // namespace

namespace sq {
// The kernel-event profile for the batched solver (batch.cu): one class for
// the kernels of its inner iterations, and a way to keep the profile out of a
// graph capture.
size_t profile_begin_batch_inner(cudaStream_t s) { return prof_begin(PC_BATCH_INNER, s); }
size_t profile_begin_batch_loop(cudaStream_t s) { return prof_begin(PC_BATCH_LOOP, s); }
void profile_end(size_t i, cudaStream_t s) { prof_end(i, s); }
bool profile_enabled() { return g_prof.on; }
bool profile_pause(bool pause) {
  static bool saved = false;
  if (pause) {
    saved = g_prof.on;
    g_prof.on = false;
  } else {
    g_prof.on = saved;
  }
  return saved;
}
static int g_inner_tol_exp = 5;
int set_inner_tol_exp(int e) {
  if (e < 2 || e > 7) return 1;
  g_inner_tol_exp = e;
  return 0;
}
double inner_tol() { return std::pow(10.0, -(double)g_inner_tol_exp); }
static int g_stage_wait_polls = 1 << 22;
int set_stage_wait_polls(int polls) {
  if (polls < 0 || polls > (1 << 24)) return 1;
  g_stage_wait_polls = polls;
  return 0;
}
int stage_wait_polls() { return g_stage_wait_polls; }
bool grid_size_ok(int N) { return valid_N(N); }
void exp_sum_nodes(int N, int R, int dim, std::vector<double> &t, std::vector<double> &w) {
  rank_r_nodes(N, R, t, w, dim);
}
int radix_plan_of(int N, int *rad) { return radix_plan(N, rad); }
int coeffs_view(const sq_coeffs *c, CellsDev *out) {
  if (!c || !out) return SQ_EINVAL;
  *out = cells_dev(c);
  return SQ_OK;
}
int precond_spec32(const sq_precond *p, SpectralDev *out, int *N) {
  if (!p || !out || !N) return SQ_EINVAL;
  *out = p->sp32;
  *N = p->N;
  return SQ_OK;
}
}  // namespace sq

// =================================================================== C ABI
extern "C" {

const char *sq_strerror(int st) {
  switch (st) {
    case SQ_OK: return "ok";
    case SQ_EINVAL: return "invalid argument";
    case SQ_ENOMEM: return "out of memory";
    case SQ_ECUDA: return "CUDA error";
    case SQ_ENOCONV: return "not converged within max_iter";
    case SQ_ETIMEOUT: return "bounded device wait timed out";
    case SQ_EBADGUESS: return "initial guess rejected";
    default: return "unknown status";
  }
}

int sq_build_coeffs(int L, int n, uint64_t seed, double p_hi, double a_lo, double a_hi, sq_stream_t stream,
                    sq_coeffs **out) {
  if (!(p_hi >= 0.0 && p_hi <= 1.0)) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = alloc_coeffs(L, n, a_lo, a_hi, s, out);
  if (st != SQ_OK) return st;
  const uint64_t thr[3] = {(uint64_t)(p_hi * 9007199254740992.0), 0, 0};  // floor(p_hi * 2^53)
  const size_t pi = prof_begin(PC_COEFF, s);
  const cudaError_t ge = launch_coeff_gen((*out)->d_phase, L, seed, thr, s);
  prof_end(pi, s);
  if (ge != cudaSuccess) {
    sq_coeffs_destroy(*out);
    *out = nullptr;
    return SQ_ECUDA;
  }
  return SQ_OK;
}

int sq_coeffs_from_host(int L, int n, const uint8_t *host_phase, double a_lo, double a_hi, sq_stream_t stream,
                        sq_coeffs **out) {
  if (!host_phase) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = alloc_coeffs(L, n, a_lo, a_hi, s, out);
  if (st != SQ_OK) return st;
  const size_t nc = (size_t)L * L * L;
  std::vector<uint8_t> norm(nc);
  for (size_t i = 0; i < nc; ++i) norm[i] = host_phase[i] ? 1 : 0;
  if (cudaMemcpyAsync((*out)->d_phase, norm.data(), nc, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    sq_coeffs_destroy(*out);
    *out = nullptr;
    return SQ_ECUDA;
  }
  return SQ_OK;
}

int sq_coeffs_regenerate(sq_coeffs *c, uint64_t seed, double p_hi, sq_stream_t stream) {
  if (!c || !(p_hi >= 0.0 && p_hi <= 1.0)) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t thr[3] = {(uint64_t)(p_hi * 9007199254740992.0), 0, 0};
  SQ_LAUNCH(PC_COEFF, s, launch_coeff_gen(c->d_phase, c->L, seed, thr, s));
  return SQ_OK;
}

// Level thresholds: tail probabilities P_m = probs[m] + ... + probs[K-1],
// summed in FP64 from the top level down, T_m = floor(min(P_m, 1) * 2^53).
static int level_thresholds(int K, const double *probs, uint64_t *thr) {
  if (K < 2 || K > kMaxLevels || !probs) return SQ_EINVAL;
  double total = 0.0;
  for (int m = 0; m < K; ++m) {
    if (!(probs[m] >= 0.0 && probs[m] <= 1.0)) return SQ_EINVAL;
    total += probs[m];
  }
  if (std::fabs(total - 1.0) > 1e-9) return SQ_EINVAL;
  thr[0] = thr[1] = thr[2] = 0;
  double tail = 0.0;
  for (int m = K - 1; m >= 1; --m) {
    tail = probs[m] + tail;
    thr[m - 1] = (uint64_t)((tail < 1.0 ? tail : 1.0) * 9007199254740992.0);
  }
  return SQ_OK;
}

// K in [2, kMaxLevels] coefficient values, each positive and finite.
static bool valid_level_values(int K, const double *values) {
  if (K < 2 || K > kMaxLevels || !values) return false;
  for (int l = 0; l < K; ++l)
    if (!(values[l] > 0.0) || !std::isfinite(values[l])) return false;
  return true;
}

int sq_coeffs_set_levels(sq_coeffs *c, int K, const double *values) {
  if (!c || !valid_level_values(K, values)) return SQ_EINVAL;
  c->levels = K;
  c->a_lo = values[0];
  c->a_hi = values[1];
  for (int l = 0; l < kMaxLevels - 2; ++l) c->a_up[l] = (l + 2 < K) ? values[l + 2] : 0.0;
  return SQ_OK;
}

int sq_build_coeffs_levels(int L, int n, uint64_t seed, int K, const double *probs, const double *values,
                           sq_stream_t stream, sq_coeffs **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  uint64_t thr[3];
  if (level_thresholds(K, probs, thr) != SQ_OK || !valid_level_values(K, values)) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = alloc_coeffs(L, n, values[0], values[1], s, out);
  if (st != SQ_OK) return st;
  st = sq_coeffs_set_levels(*out, K, values);
  if (st == SQ_OK) {
    const size_t pi = prof_begin(PC_COEFF, s);
    if (launch_coeff_gen((*out)->d_phase, L, seed, thr, s) != cudaSuccess) st = SQ_ECUDA;
    prof_end(pi, s);
  }
  if (st != SQ_OK) {
    sq_coeffs_destroy(*out);
    *out = nullptr;
  }
  return st;
}

int sq_coeffs_from_host_levels(int L, int n, const uint8_t *host_level, int K, const double *values,
                               sq_stream_t stream, sq_coeffs **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (!host_level || !valid_level_values(K, values)) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int st = alloc_coeffs(L, n, values[0], values[1], s, out);
  if (st != SQ_OK) return st;
  st = sq_coeffs_set_levels(*out, K, values);
  if (st == SQ_OK) {
    const size_t nc = (size_t)L * L * L;
    std::vector<uint8_t> lv(nc);  // levels past the top one read as the top level
    for (size_t i = 0; i < nc; ++i) lv[i] = host_level[i] < K ? host_level[i] : (uint8_t)(K - 1);
    if (cudaMemcpyAsync((*out)->d_phase, lv.data(), nc, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = SQ_ECUDA;
  }
  if (st != SQ_OK) {
    sq_coeffs_destroy(*out);
    *out = nullptr;
  }
  return st;
}

int sq_coeffs_regenerate_levels(sq_coeffs *c, uint64_t seed, int K, const double *probs, sq_stream_t stream) {
  uint64_t thr[3];
  if (!c || K != c->levels || level_thresholds(K, probs, thr) != SQ_OK) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SQ_LAUNCH(PC_COEFF, s, launch_coeff_gen(c->d_phase, c->L, seed, thr, s));
  return SQ_OK;
}

int sq_coeffs_upload(sq_coeffs *c, const uint8_t *host_phase, sq_stream_t stream) {
  if (!c || !host_phase) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SQ_CK(cudaMemcpyAsync(c->d_phase, host_phase, (size_t)c->L * c->L * c->L, cudaMemcpyHostToDevice, s));
  return SQ_OK;
}

int sq_profile_enable(int enable) {
  g_prof.on = enable != 0;
  if (g_prof.on) {
    g_prof.used = 0;
    g_prof.cls.clear();
  }
  return SQ_OK;
}

int sq_profile_read(double *ms, int64_t *launches, int max_classes) {
  double acc[PC_COUNT] = {0};
  int64_t cnt[PC_COUNT] = {0};
  std::vector<float> times[PC_COUNT];
  for (size_t k = 0; k < g_prof.cls.size(); ++k) {
    const size_t i = 2 * k;
    if (cudaEventSynchronize(g_prof.pool[i + 1]) != cudaSuccess) return -SQ_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, g_prof.pool[i], g_prof.pool[i + 1]) != cudaSuccess) return -SQ_ECUDA;
    acc[g_prof.cls[k]] += t;
    cnt[g_prof.cls[k]] += 1;
    times[g_prof.cls[k]].push_back(t);
  }
  // launches that did work: at least half of the class median (the
  // others returned at entry because the solve had already stopped)
  for (int k = 0; k < PC_COUNT; ++k) {
    g_prof_work_ms[k] = 0.0;
    g_prof_work_n[k] = 0;
    if (times[k].empty()) continue;
    std::vector<float> v = times[k];
    std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
    const float thr = 0.5f * v[v.size() / 2];
    for (float t : times[k])
      if (t >= thr) {
        g_prof_work_ms[k] += t;
        g_prof_work_n[k] += 1;
      }
  }
  for (int k = 0; k < PC_COUNT && k < max_classes; ++k) {
    if (ms) ms[k] = acc[k];
    if (launches) launches[k] = cnt[k];
  }
  g_prof.used = 0;
  g_prof.cls.clear();
  return PC_COUNT;
}

int sq_profile_work(double *ms, int64_t *launches, int max_classes) {
  for (int k = 0; k < PC_COUNT && k < max_classes; ++k) {
    if (ms) ms[k] = g_prof_work_ms[k];
    if (launches) launches[k] = g_prof_work_n[k];
  }
  return PC_COUNT;
}

const char *sq_profile_class_name(int k) { return (k >= 0 && k < PC_COUNT) ? kProfNames[k] : "?"; }

int64_t sq_launch_count(void) { return g_launches; }

int sq_coeffs_set_subcell(sq_coeffs *c, int sub) {
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

int sq_coeffs_cells(const sq_coeffs *c, uint8_t *host_phase, int64_t *n_hi) {
  if (!c) return SQ_EINVAL;
  const size_t nc = (size_t)c->L * c->L * c->L;
  std::vector<uint8_t> tmp(nc);
  SQ_CK(cudaMemcpyAsync(tmp.data(), c->d_phase, nc, cudaMemcpyDeviceToHost, c->stream));
  SQ_CK(cudaStreamSynchronize(c->stream));
  if (host_phase) std::memcpy(host_phase, tmp.data(), nc);
  if (n_hi) {
    int64_t k = 0;
    for (size_t i = 0; i < nc; ++i) k += tmp[i] ? 1 : 0;
    *n_hi = k;
  }
  return SQ_OK;
}

int sq_coeffs_shape(const sq_coeffs *c, int *L, int *n, int *N) {
  if (!c) return SQ_EINVAL;
  if (L) *L = c->L;
  if (n) *n = c->n;
  if (N) *N = c->N;
  return SQ_OK;
}

void sq_coeffs_destroy(sq_coeffs *c) {
  if (!c) return;
  if (c->d_phase) cudaFree(c->d_phase);
  if (c->d_st) cudaFree(c->d_st);
  if (c->d_partials) cudaFree(c->d_partials);
  if (c->h_st) cudaFreeHost(c->h_st);
  delete c;
}

}  // extern "C"

namespace sq {

// Uploads a preconditioner: rank R >= 0 canonical terms with the host
// factors f (3 x R x N, axis a of term r at f + (a R + r) N; unscaled, so
// that G(k) = sum_r f1_r(k1) f2_r(k2) f3_r(k3)); R = 0 is the exact diagonal.
// t, w: the exponential-sum nodes and weights when the factors come from one.
// The multiplier tables of pass C (SpectralDev::gtab): G at every
// mirror-reduced mode (m1, m2, m3), m <= N/2, summed in FP64 from the scaled
// factors (or scale / (l1 + l2 + l3) for the exact diagonal); G(0,0,0) = 0.
// They hold G times the factor pass C would otherwise apply per mode (exact
// powers of 2): FP64 8 G (the complex x2 route), indexed by (m1, m2, m3); FP32
// 2 G (the Hartley route) by (m1, m2, k3) with k3 over the whole axis (each
// FP32 tile prefetches its 2P columns into shared memory).
__global__ void k_build_gtab(int N, int R, const double *lam, const double *u, double scale, double *g64,
                             float *g32) {
  const int H = N / 2 + 1;
  const size_t n = (size_t)H * H * H;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int m3 = (int)(i % H), m2 = (int)((i / H) % H), m1 = (int)(i / ((size_t)H * H));
    double g = 0.0;
    if (m1 != 0 || m2 != 0 || m3 != 0) {
      if (R == 0) {
        g = scale / (lam[m1] + lam[m2] + lam[m3]);
      } else {
        for (int r = 0; r < R; ++r)
          g = fma(u[(size_t)r * N + m1], u[(size_t)(R + r) * N + m2] * u[(size_t)(2 * R + r) * N + m3], g);
      }
    }
    g64[i] = 8.0 * g;
    const size_t row = ((size_t)m1 * H + m2) * N;
    g32[row + m3] = (float)(2.0 * g);
    if (m3 != 0 && m3 != N - m3) g32[row + N - m3] = (float)(2.0 * g);
  }
}

int precond_create(int N, int R, const double *f, const std::vector<double> &t, const std::vector<double> &w,
                   sq_precond **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (!valid_N(N) || R < 0 || R > kMaxRank || (R > 0 && !f)) return SQ_EINVAL;
  const double pi = 3.14159265358979323846;
  std::vector<double> tw64(2 * N), lam64(N), u64((size_t)3 * (R > 0 ? R : 1) * N, 0.0);
  for (int m = 0; m < N; ++m) {
    const double ang = 2.0 * pi * m / N;
    tw64[2 * m] = std::cos(ang);
    tw64[2 * m + 1] = -std::sin(ang);
    const double sn = std::sin(pi * m / N);
    lam64[m] = 4.0 * sn * sn;
  }
  const double fold = 1.0 / (4.0 * N);  // (64 N^3)^(-1/3)
  for (size_t i = 0; i < (size_t)3 * R * N; ++i) u64[i] = f[i] * fold;
  std::vector<float> tw32(2 * N), lam32(N), u32(u64.size());
  for (size_t i = 0; i < tw64.size(); ++i) tw32[i] = (float)tw64[i];
  for (int i = 0; i < N; ++i) lam32[i] = (float)lam64[i];
  for (size_t i = 0; i < u64.size(); ++i) u32[i] = (float)u64[i];

  sq_precond *pc = new (std::nothrow) sq_precond();
  if (!pc) return SQ_ENOMEM;
  pc->N = N;
  pc->rank = R;
  pc->t = t;
  pc->w = w;
  if (R > 0) pc->f.assign(f, f + (size_t)3 * R * N);
  const size_t b_tw64 = tw64.size() * 8, b_lam64 = lam64.size() * 8, b_u64 = u64.size() * 8;
  const size_t b_tw32 = tw32.size() * 4, b_lam32 = lam32.size() * 4, b_u32 = u32.size() * 4;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t H = (size_t)N / 2 + 1;
  const bool with_tab = N <= kGtabMaxN;
  const size_t b_g64 = with_tab ? H * H * H * 8 : 0, b_g32 = with_tab ? H * H * (size_t)N * 4 : 0;
  const size_t total =
      al(b_tw64) + al(b_lam64) + al(b_u64) + al(b_tw32) + al(b_lam32) + al(b_u32) + al(b_g64) + al(b_g32);
  if (cudaMalloc(&pc->d_mem, total) != cudaSuccess) {
    delete pc;
    return SQ_ENOMEM;
  }
  char *bp = static_cast<char *>(pc->d_mem);
  char *p_tw64 = bp;
  char *p_lam64 = p_tw64 + al(b_tw64);
  char *p_u64 = p_lam64 + al(b_lam64);
  char *p_tw32 = p_u64 + al(b_u64);
  char *p_lam32 = p_tw32 + al(b_tw32);
  char *p_u32 = p_lam32 + al(b_lam32);
  char *p_g64 = p_u32 + al(b_u32);
  char *p_g32 = p_g64 + al(b_g64);
  if (cudaMemcpy(p_tw64, tw64.data(), b_tw64, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p_lam64, lam64.data(), b_lam64, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p_u64, u64.data(), b_u64, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p_tw32, tw32.data(), b_tw32, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p_lam32, lam32.data(), b_lam32, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p_u32, u32.data(), b_u32, cudaMemcpyHostToDevice) != cudaSuccess) {
    sq_precond_destroy(pc);
    return SQ_ECUDA;
  }
  SpectralDev sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.N = N;
  sp.rank = R;
  sp.nst = radix_plan(N, sp.radix);
  sp.scale = 1.0 / (64.0 * (double)N * N * N);
  if (with_tab) {
    k_build_gtab<<<1024, 256>>>(N, R, reinterpret_cast<const double *>(p_lam64),
                                reinterpret_cast<const double *>(p_u64), sp.scale, reinterpret_cast<double *>(p_g64),
                                reinterpret_cast<float *>(p_g32));
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
      sq_precond_destroy(pc);
      return SQ_ECUDA;
    }
  }
  pc->sp64 = sp;
  pc->sp64.tw = p_tw64;
  pc->sp64.lam = p_lam64;
  pc->sp64.u = p_u64;
  pc->sp64.gtab = with_tab ? p_g64 : nullptr;
  pc->sp32 = sp;
  pc->sp32.tw = p_tw32;
  pc->sp32.lam = p_lam32;
  pc->sp32.u = p_u32;
  pc->sp32.gtab = with_tab ? p_g32 : nullptr;
  *out = pc;
  return SQ_OK;
}

}  // namespace sq

extern "C" {

int sq_precond_setup(int N, int rank, sq_precond **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (!valid_N(N) || rank < 0 || rank == 1 || rank > kMaxExpRank) return SQ_EINVAL;
  std::vector<double> t, w, f;
  if (rank > 0) {
    // the same exponential-sum factor u_r(k) = w_r^(1/3) exp(-t_r lambda_k) on every axis
    rank_r_nodes(N, rank, t, w);
    f.resize((size_t)3 * rank * N);
    for (int r = 0; r < rank; ++r) {
      const double wr = std::cbrt(w[r]);
      for (int k = 0; k < N; ++k) {
        const double sn = std::sin(3.14159265358979323846 * k / N);
        const double v = wr * std::exp(-t[r] * 4.0 * sn * sn);
        for (int a = 0; a < 3; ++a) f[((size_t)a * rank + r) * N + k] = v;
      }
    }
  }
  return precond_create(N, rank, f.data(), t, w, out);
}

// max over nonzero modes of |g G(k) - 1|, g = lambda_k1 + lambda_k2 +
// lambda_k3, over k in [0, N/2]^3 (every factor is even).
static double precond_max_rel_err(const sq_precond *p) {
  const int N = p->N, M = N / 2 + 1, R = p->rank;
  std::vector<double> lam(M);
  for (int m = 0; m < M; ++m) {
    const double sn = std::sin(3.14159265358979323846 * m / N);
    lam[m] = 4.0 * sn * sn;
  }
  double worst = 0.0;
  std::vector<double> v23((size_t)R);
  for (int k2 = 0; k2 < M; ++k2)
    for (int k3 = 0; k3 < M; ++k3) {
      for (int r = 0; r < R; ++r)
        v23[r] = p->f[((size_t)1 * R + r) * N + k2] * p->f[((size_t)2 * R + r) * N + k3];
      for (int k1 = 0; k1 < M; ++k1) {
        const double g = lam[k1] + lam[k2] + lam[k3];
        if (!(g > 0.0)) continue;
        double G = 0.0;
        if (R == 0) {
          G = 1.0 / g;
        } else {
          for (int r = 0; r < R; ++r) G += p->f[(size_t)r * N + k1] * v23[r];
        }
        worst = std::max(worst, std::fabs(g * G - 1.0));
      }
    }
  return worst;
}

int sq_precond_info(const sq_precond *p, int *rank, double *max_rel_err) {
  if (!p) return SQ_EINVAL;
  if (rank) *rank = p->rank;
  if (max_rel_err) *max_rel_err = precond_max_rel_err(p);
  return SQ_OK;
}

int sq_set_tiles(const sq_tile_config *tiles, int ntiles) {
  if (ntiles < 0 || (ntiles > 0 && !tiles)) return SQ_EINVAL;
  ++g_option_epoch;  // launch parameters may change: no stored iteration graph applies
  for (int k = 0; k < ntiles; ++k) {
    const int N = tiles[k].N;
    if (!valid_N(N)) return SQ_EINVAL;
    // an entry sets every field of its grid size, 0 restoring the default
    if (set_dht_pencils_override(N, tiles[k].dht_pencils) != 0) return SQ_EINVAL;
    if (set_stencil_planes_override(N, tiles[k].stencil_planes) != 0) return SQ_EINVAL;
    if (set_stencil_rows_override(N, tiles[k].stencil_rows) != 0) return SQ_EINVAL;
    if (set_dht_pencils_e_override(N, tiles[k].dht_pencils_e) != 0) return SQ_EINVAL;
  }
  if (ntiles == 0) {
    for (int N = 8; N <= kMaxN; ++N) {
      set_dht_pencils_override(N, 0);
      set_dht_pencils_e_override(N, 0);
      set_stencil_planes_override(N, 0);
      set_stencil_rows_override(N, 0);
    }
  }
  return SQ_OK;
}

int sq_set_option(int key, int value) {
  ++g_option_epoch;  // launch parameters may change: no stored iteration graph applies
  if (key == SQ_OPT_PCG_GRAPHS) {
    if (value < 0 || value > 1) return SQ_EINVAL;
    g_pcg_graphs = value;
    return SQ_OK;
  }
  if (key == SQ_OPT_STRIDED_TWO_STAGE) return set_strided_fast(value) == 0 ? SQ_OK : SQ_EINVAL;
  if (key == SQ_OPT_STENCIL_ROWS) return set_stencil_rows(value) == 0 ? SQ_OK : SQ_EINVAL;
  if (key == SQ_OPT_INNER_TOL_EXP) return set_inner_tol_exp(value) == 0 ? SQ_OK : SQ_EINVAL;
  if (key == SQ_OPT_WAIT_POLLS) return set_stage_wait_polls(value) == 0 ? SQ_OK : SQ_EINVAL;
  if (key == SQ_OPT_MULTIPLIER_TABLE) return set_use_gtab(value) == 0 ? SQ_OK : SQ_EINVAL;
  if (key == SQ_OPT_CONV_TC) return set_conv_tc(value) == 0 ? SQ_OK : SQ_EINVAL;
  return SQ_EINVAL;
}

int sq_precond_factors(const sq_precond *p, double *t, double *w) {
  if (!p || (int)p->t.size() != p->rank) return SQ_EINVAL;  // not an exponential sum
  for (int r = 0; r < p->rank; ++r) {
    if (t) t[r] = p->t[r];
    if (w) w[r] = p->w[r];
  }
  return SQ_OK;
}

void sq_precond_destroy(sq_precond *p) {
  if (!p) return;
  if (p->d_mem) cudaFree(p->d_mem);
  delete p;
}

int sq_workspace_create(int N, int precision, sq_workspace **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (!valid_N(N) || (precision != SQ_FP64 && precision != SQ_FP32_REFINE)) return SQ_EINVAL;
  sq_workspace *w = new (std::nothrow) sq_workspace();
  if (!w) return SQ_ENOMEM;
  w->N = N;
  w->precision = precision;
  const size_t n3 = (size_t)N * N * N;
  bool ok = true;
  if (precision == SQ_FP64)
    ok = ok && cudaMalloc(&w->f64, sizeof(double) * 4 * n3) == cudaSuccess;
  else
    ok = ok && cudaMalloc(&w->f32, sizeof(float) * 5 * n3) == cudaSuccess;
  ok = ok && cudaMalloc(&w->d_st, 2 * sizeof(Scalars)) == cudaSuccess;
  ok = ok && cudaMalloc(&w->d_partials, sizeof(double) * kMaxQ * kMaxPartials) == cudaSuccess;
  ok = ok && cudaMallocHost(&w->h_st, 2 * sizeof(Scalars)) == cudaSuccess;
  ok = ok && cudaMallocHost(&w->h_poll, 2 * sizeof(int)) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&w->ev[0], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaEventCreateWithFlags(&w->ev[1], cudaEventDisableTiming) == cudaSuccess;
  if (ok) ok = cudaMemset(w->d_st, 0, 2 * sizeof(Scalars)) == cudaSuccess;
  if (!ok) {
    sq_workspace_destroy(w);
    return SQ_ENOMEM;
  }
  *out = w;
  return SQ_OK;
}

void sq_workspace_destroy(sq_workspace *w) {
  if (!w) return;
  if (w->f64) cudaFree(w->f64);
  if (w->f32) cudaFree(w->f32);
  if (w->d_st) cudaFree(w->d_st);
  if (w->d_partials) cudaFree(w->d_partials);
  if (w->h_st) cudaFreeHost(w->h_st);
  if (w->h_poll) cudaFreeHost(w->h_poll);
  if (w->ev[0]) cudaEventDestroy(w->ev[0]);
  if (w->ev[1]) cudaEventDestroy(w->ev[1]);
  for (sq_workspace::IterGraph &e : w->graphs) {
    cudaGraphExecDestroy(e.exec);
    cudaGraphDestroy(e.graph);
  }
  delete w;
}

int sq_pcg_solve(const sq_coeffs *c, const sq_precond *pc, sq_workspace *w, int dir, double tol, int max_iter,
                 int precision, const double *x0, double *psi, sq_solve_info *info, sq_stream_t stream) {
  if (!c || !pc || !w || !psi) return SQ_EINVAL;
  if (dir < 0 || dir > 2 || !(tol > 0.0) || max_iter < 1) return SQ_EINVAL;
  if (pc->N != c->N || w->N != c->N || w->precision != precision) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (info) std::memset(info, 0, sizeof(*info));
  if (precision == SQ_FP64) return solve_fp64(c, pc, w, dir, tol, max_iter, x0, psi, info, s);
  if (precision == SQ_FP32_REFINE) return solve_fp32_refine(c, pc, w, dir, tol, max_iter, x0, psi, info, s);
  return SQ_EINVAL;
}

int sq_homogenized_matrix(const sq_coeffs *c, const double *psi0, const double *psi1, const double *psi2,
                          double *A_hom, double *A_energy, sq_stream_t stream) {
  if (!c || !psi0 || !psi1 || !psi2 || !A_hom) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const RedBuf rb = redbuf<double>(c->d_st, c->d_partials);
  SQ_LAUNCH(PC_AHOM, s, launch_ahom(cells_dev(c), psi0, psi1, psi2, rb, A_energy != nullptr, s));
  int st = read_scalars(c->h_st, c->d_st, s);
  if (st != SQ_OK) return st;
  const double nn = (double)c->N * c->N * c->N;
  const double *red = c->h_st->red;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A_hom[3 * i + j] = ((i == j) ? red[9 + j] : 0.0) / nn + red[3 * i + j] / nn;
  if (A_energy) {
    const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A_energy[3 * i + j] = red[12 + idx[i][j]] / nn;
  }
  return SQ_OK;
}

int sq_apply_operator(const sq_coeffs *c, const double *x, double *y, sq_stream_t stream) {
  if (!c || !x || !y || x == y) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SQ_LAUNCH(PC_MATVEC, s, (launch_stencil<double, double>(cells_dev(c), ST_MATVEC, 0, x, y, redbuf<double>(c->d_st, c->d_partials),
                                        FIN_NONE, false, s)));
  return SQ_OK;
}

int sq_apply_operator_f32(const sq_coeffs *c, const float *x, float *y, sq_stream_t stream) {
  if (!c || !x || !y || x == y) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SQ_LAUNCH(PC_MATVEC, s, (launch_stencil<float, float>(cells_dev(c), ST_MATVEC, 0, x, y, redbuf<float>(c->d_st, c->d_partials),
                                      FIN_NONE, false, s)));
  return SQ_OK;
}

int sq_rhs(const sq_coeffs *c, int dir, double *b, sq_stream_t stream) {
  if (!c || !b || dir < 0 || dir > 2) return SQ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SQ_LAUNCH(PC_RESID, s, (launch_stencil<double, double>(cells_dev(c), ST_RHS, dir, nullptr, b, redbuf<double>(c->d_st, c->d_partials),
                                        FIN_NONE, false, s)));
  return SQ_OK;
}

int sq_apply_precond(const sq_precond *pc, sq_workspace *w, const double *r, double *z, sq_stream_t stream) {
  if (!pc || !w || !r || !z || w->N != pc->N || w->precision != SQ_FP64) return SQ_EINVAL;
  const size_t n3 = (size_t)pc->N * pc->N * pc->N;
  return apply_precond_t<double>(pc, w, r, z, w->f64 + 3 * n3, reinterpret_cast<cudaStream_t>(stream));
}

int sq_apply_precond_f32(const sq_precond *pc, sq_workspace *w, const float *r, float *z, sq_stream_t stream) {
  if (!pc || !w || !r || !z || w->N != pc->N || w->precision != SQ_FP32_REFINE) return SQ_EINVAL;
  const size_t n3 = (size_t)pc->N * pc->N * pc->N;
  return apply_precond_t<float>(pc, w, r, z, w->f32 + 3 * n3, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
