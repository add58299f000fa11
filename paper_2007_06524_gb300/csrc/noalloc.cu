// Homogenized matrix for callers that cannot allocate device memory.
//
// Who needs this: code that runs while its stream is being captured into a
// CUDA graph (the runtime allocator may not be called during capture), and
// host frameworks that own every byte of device memory through their own
// fixed pool and do not allow library code to call cudaMalloc/cudaFree. Such a
// caller can still ask for A_hom: it passes the cell phases, the three
// correctors and an 18-double output buffer, all in device memory it already
// owns, and the reduction scratch comes from a file-scope __device__ array of
// this library instead of an allocation.
//
// Limits and sharing:
//  * the scratch holds kNoAllocScratchDoubles doubles (2.36 MB); every GPU that
//    loads libsq keeps it until the process exits;
//  * grids up to N = L*n = 512 (the library's limit), so the reduction never
//    uses more than kMaxPartials blocks; larger or malformed sizes are
//    rejected with SQ_EINVAL;
//  * all calls on one device share the one array and it keeps the contents of
//    the last call; the only value that must start at zero (the last-block
//    counter) is cleared at the start of every call. Calls that overlap on the
//    GPU (two streams, or two host threads) race on the array and give wrong
//    results: order them on one stream;
//  * the first call on each device looks up the array's device address with
//    cudaGetSymbolAddress while that device is current; make that first call
//    before any stream capture begins.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace sq {

namespace {

// Scalars block first (512 bytes reserved), then the per-block partials laid
// out as reduce_last_block expects: quantity q of block b at q * kMaxPartials + b.
constexpr size_t kScalarsDoubles = 64;
constexpr int kAhomQ = 18;
constexpr size_t kNoAllocScratchDoubles = kScalarsDoubles + (size_t)kAhomQ * kMaxPartials;
static_assert(sizeof(Scalars) <= kScalarsDoubles * sizeof(double), "scalars block too small");

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch on the current device (looked up once per device).
int scratch_address(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SQ_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return SQ_EINVAL;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SQ_ECUDA;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
  return SQ_OK;
}

bool grid_ok(int L, int n) {
  if (L < 1 || n < 2) return false;
  const long long N = (long long)L * n;
  if (N < 8 || N > kMaxN || (N & 1)) return false;
  long long m = N;
  while (m % 2 == 0) m /= 2;
  if (m % 3 == 0) m /= 3;
  return m == 1;
}

// A_hom (edge form, 9 values) and the energy form (9 values) from the sums the
// reduction left in st->red: 0..8 sum a_j D_j psi_i, 9..11 sum a_j, 12..17 the
// energy sums for (00,01,02,11,12,22).
__global__ void k_ahom_finish(const double *scratch, double nn, double *out) {
  const Scalars *st = reinterpret_cast<const Scalars *>(scratch);
  const int t = threadIdx.x;
  if (t < 9) {
    const int i = t / 3, j = t % 3;
    out[t] = ((i == j) ? st->red[9 + j] : 0.0) / nn + st->red[3 * i + j] / nn;
  } else if (t < 18) {
    const int e = t - 9, i = e / 3, j = e % 3;
    const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    out[t] = st->red[12 + idx[i][j]] / nn;
  }
}

}  // namespace
}  // namespace sq

using namespace sq;

extern "C" int sq_homogenized_matrix_noalloc(int L, int n, const uint8_t *phase, double a_lo, double a_hi,
                                             const double *psi0, const double *psi1, const double *psi2,
                                             double *out, sq_stream_t stream) {
  if (!grid_ok(L, n) || !phase || !psi0 || !psi1 || !psi2 || !out) return SQ_EINVAL;
  if (!(a_lo > 0.0) || !(a_hi > 0.0) || !std::isfinite(a_lo) || !std::isfinite(a_hi)) return SQ_EINVAL;
  double *scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st != SQ_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Scalars *sc = reinterpret_cast<Scalars *>(scratch);
  if (cudaMemsetAsync(&sc->ticket, 0, sizeof(sc->ticket), s) != cudaSuccess) return SQ_ECUDA;
  CellsDev c;
  c.phase = phase;
  c.L = L;
  c.n = n;
  c.N = L * n;
  c.a_lo = a_lo;
  c.a_hi = a_hi;
  fill_tables(c);
  RedBuf rb;
  rb.st = sc;
  rb.partials = scratch + kScalarsDoubles;
  if (launch_ahom(c, psi0, psi1, psi2, rb, true, s) != cudaSuccess) return SQ_ECUDA;
  const double nn = (double)c.N * c.N * c.N;
  k_ahom_finish<<<1, 32, 0, s>>>(scratch, nn, out);
  if (cudaGetLastError() != cudaSuccess) return SQ_ECUDA;
  return SQ_OK;
}
