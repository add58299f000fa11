// Ensemble statistics of the homogenized matrix (Sec. 5, "Example of
// application to numerical estimation of the homogenized coefficient
// matrix"). For M realizations of the L^3 checkerboard at one period L, the
// three correctors of every realization are solved together in batches
// (FP32 PCG in FP64 refinement, one batched launch per kernel for the whole
// chunk), the edge-form A_hom of each realization follows (Eq. 21 on the
// grid), and the host forms, entry-wise in FP64 and in realization order,
//   the empirical average  A^M_L = (1/M) sum_m A^(m)_L        (Eq. A_hom_Empir)
//   sigma^M_L = sqrt( sum_m (A^(m)_L - A^M_L)^2 / (M - 1) ),
// the computable estimate of sigma_L, which Eq. var bounds by C L^{-d/2}.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "sq.h"

extern "C" int sq_ensemble_ahom(int L, int n, const uint64_t *seeds, int M, double p_hi, double a_lo,
                                double a_hi, int rank, double tol, int max_iter, int chunk, double *mean,
                                double *sigma, double *per_real, int *iters, sq_stream_t stream) {
  if (!seeds || M < 2 || !mean || !sigma || chunk < 0 || !(tol > 0.0) || max_iter < 1 || L < 1 || n < 2)
    return SQ_EINVAL;
  const int N = L * n;
  sq_precond *pc = nullptr;
  int st = sq_precond_setup(N, rank, &pc);
  if (st != SQ_OK) return st;
  const int C = (chunk == 0 || chunk > M) ? M : chunk;
  const size_t n3 = (size_t)N * N * N;
  double *psi = nullptr;  // the three correctors of every realization of a chunk
  if (cudaMalloc(&psi, sizeof(double) * 3 * n3 * (size_t)C) != cudaSuccess) {
    sq_precond_destroy(pc);
    return SQ_ENOMEM;
  }
  std::vector<double> A((size_t)M * 9);
  std::vector<sq_coeffs *> cs(C, nullptr);
  std::vector<sq_solve_desc> descs(3 * (size_t)C);
  std::vector<const sq_precond *> precs(3 * (size_t)C, pc);
  std::vector<sq_solve_info> infos(3 * (size_t)C);
  bool noconv = false;
  for (int m0 = 0; m0 < M && st == SQ_OK; m0 += C) {
    const int cnt = std::min(C, M - m0);
    for (int k = 0; k < cnt && st == SQ_OK; ++k)
      st = sq_build_coeffs(L, n, seeds[m0 + k], p_hi, a_lo, a_hi, stream, &cs[k]);
    if (st == SQ_OK) {
      for (int k = 0; k < cnt; ++k)
        for (int i = 0; i < 3; ++i) {
          sq_solve_desc &d = descs[3 * (size_t)k + i];
          d.coeffs = cs[k];
          d.dir = i;
          d.psi = psi + (3 * (size_t)k + i) * n3;
        }
      sq_batch *b = nullptr;
      st = sq_batch_create(3 * cnt, descs.data(), precs.data(), nullptr, 0, &b);
      if (st == SQ_OK) {
        const int sb = sq_pcg_solve_batched(b, tol, max_iter, infos.data(), stream);
        if (sb == SQ_ENOCONV)
          noconv = true;
        else
          st = sb;
        sq_batch_destroy(b);
      }
    }
    for (int k = 0; k < cnt && st == SQ_OK; ++k)
      st = sq_homogenized_matrix(cs[k], psi + 3 * (size_t)k * n3, psi + (3 * (size_t)k + 1) * n3,
                                 psi + (3 * (size_t)k + 2) * n3, &A[(size_t)(m0 + k) * 9], nullptr, stream);
    if (st == SQ_OK && iters)
      for (int k = 0; k < 3 * cnt; ++k) iters[3 * (size_t)m0 + k] = infos[k].iters;
    for (int k = 0; k < cnt; ++k) {
      sq_coeffs_destroy(cs[k]);
      cs[k] = nullptr;
    }
  }
  cudaFree(psi);
  sq_precond_destroy(pc);
  if (st != SQ_OK) return st;
  for (int e = 0; e < 9; ++e) {
    double s = 0.0;
    for (int m = 0; m < M; ++m) s += A[(size_t)m * 9 + e];
    mean[e] = s / M;
    double ss = 0.0;
    for (int m = 0; m < M; ++m) {
      const double d = A[(size_t)m * 9 + e] - mean[e];
      ss += d * d;
    }
    sigma[e] = std::sqrt(ss / (M - 1));
  }
  if (per_real) std::copy(A.begin(), A.end(), per_real);
  return noconv ? SQ_ENOCONV : SQ_OK;
}
