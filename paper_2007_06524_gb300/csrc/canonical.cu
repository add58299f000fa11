// Canonical preconditioners other than the exponential sum: from factors the
// caller supplies, and by the paper's own route (Sec. 4.2): a Tucker
// decomposition of G+ (Eqs. 32-33) followed by a Tucker-to-canonical
// transform of its core. Host-side setup; the factors then drive the same
// pass-C kernels as every other rank-R preconditioner.
//
// Tucker: the higher-order SVD (De Lathauwer, De Moor & Vandewalle, SIMAX
// 2000). G+ is symmetric in its three indices, so one factor U (N x r, the
// leading left singular vectors of the mode-1 unfolding) serves all modes.
// G+(k) depends on k_a only through lambda_{k_a} = lambda_{N - k_a}, so the
// rows k and N - k of the unfolding coincide and the singular vectors with
// nonzero singular values are even. The decomposition is therefore computed
// on the reduced index m = min(k, N - k) in [0, N/2] with multiplicities
// c_m (1 at m = 0 and m = N/2, else 2): the Gram matrix of the unfolding
// restricted to even vectors is D K D with D = diag(sqrt(c)) and
// K[a][b] = sum_{m2,m3} c_m2 c_m3 H(a,m2,m3) H(b,m2,m3), H the reduced
// tensor; an eigenvector y of D K D gives u(m) = y_m / sqrt(c_m).
// Core: beta = G+ x1 U^T x2 U^T x3 U^T, contracted one mode at a time.
// Tucker-to-canonical: each mode-3 slice beta[:, :, c] is symmetric; its
// eigenpairs (sigma, e) give the terms sigma (U e) (x) (U e) (x) U[:, c],
// r^2 in all; terms with |sigma| <= tol * max|sigma| are dropped.
// The eigenproblems use the cyclic Jacobi method (Jacobi 1846; rotations in
// the stable form of Rutishauser 1966).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"

namespace sq {
namespace {

// Eigen-decomposition of the symmetric n x n matrix A (row-major, destroyed):
// eigenvalues in w (descending), eigenvectors in the columns of V (row-major
// n x n).
void jacobi_eigh(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  double total = 0.0;
  for (size_t i = 0; i < (size_t)n * n; ++i) total += A[i] * A[i];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (!(off > 1e-32 * total)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        // rotation in the (p, q) plane that zeroes A[p][q]
        const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q of A J
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q of J^T (A J)
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V J
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return A[(size_t)a * n + a] > A[(size_t)b * n + b]; });
  std::vector<double> Vs((size_t)n * n);
  w.resize(n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)order[j] * n + order[j]];
    for (int i = 0; i < n; ++i) Vs[(size_t)i * n + j] = V[(size_t)i * n + order[j]];
  }
  V.swap(Vs);
}

bool even_rows(const double *f, int R, int N) {
  for (int r = 0; r < R; ++r) {
    const double *row = f + (size_t)r * N;
    double mx = 0.0;
    for (int k = 0; k < N; ++k) mx = std::max(mx, std::fabs(row[k]));
    for (int k = 1; k < N; ++k)
      if (!(std::fabs(row[k] - row[N - k]) <= 1e-12 * mx)) return false;
    for (int k = 0; k < N; ++k)
      if (!std::isfinite(row[k])) return false;
  }
  return true;
}

}  // namespace
}  // namespace sq

using namespace sq;

extern "C" {

int sq_precond_setup_canonical(int N, int R, const double *f1, const double *f2, const double *f3,
                               sq_precond **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  if (R < 1 || R > kMaxRank || !f1 || !grid_size_ok(N)) return SQ_EINVAL;
  const double *fa[3] = {f1, f2 ? f2 : f1, f3 ? f3 : f1};
  for (int a = 0; a < 3; ++a)
    if (!even_rows(fa[a], R, N)) return SQ_EINVAL;
  std::vector<double> f;
  try {
    f.resize((size_t)3 * R * N);
  } catch (...) {
    return SQ_ENOMEM;
  }
  for (int a = 0; a < 3; ++a) std::copy(fa[a], fa[a] + (size_t)R * N, f.begin() + (size_t)a * R * N);
  return precond_create(N, R, f.data(), {}, {}, out);
}

int sq_precond_setup_tucker(int N, int r, double tol, sq_precond **out) {
  if (!out) return SQ_EINVAL;
  *out = nullptr;
  const int M = N / 2 + 1;
  if (!grid_size_ok(N) || r < 1 || r > M || r > 64 || !(tol >= 0.0) || !(tol < 1.0)) return SQ_EINVAL;
  std::vector<double> lam(M), cm(M), H, K, B, y, ev, U, T1, T2, beta, f;
  try {
    for (int m = 0; m < M; ++m) {
      const double sn = std::sin(3.14159265358979323846 * m / N);
      lam[m] = 4.0 * sn * sn;
      cm[m] = (m == 0 || 2 * m == N) ? 1.0 : 2.0;
    }
    // reduced tensor H(m1, m2, m3), H(0, 0, 0) = 0 (the pseudo-inverse)
    H.resize((size_t)M * M * M);
    for (int a = 0; a < M; ++a)
      for (int b = 0; b < M; ++b)
        for (int c = 0; c < M; ++c) {
          const double g = lam[a] + lam[b] + lam[c];
          H[((size_t)a * M + b) * M + c] = (g > 0.0) ? 1.0 / g : 0.0;
        }
    // weighted Gram matrix of the mode-1 unfolding, B = D K D
    std::vector<double> wt((size_t)M * M);
    for (int b = 0; b < M; ++b)
      for (int c = 0; c < M; ++c) wt[(size_t)b * M + c] = cm[b] * cm[c];
    B.assign((size_t)M * M, 0.0);
    for (int a = 0; a < M; ++a)
      for (int a2 = a; a2 < M; ++a2) {
        const double *ha = &H[(size_t)a * M * M], *hb = &H[(size_t)a2 * M * M];
        double s = 0.0;
        for (size_t i = 0; i < (size_t)M * M; ++i) s += wt[i] * ha[i] * hb[i];
        s *= std::sqrt(cm[a] * cm[a2]);
        B[(size_t)a * M + a2] = s;
        B[(size_t)a2 * M + a] = s;
      }
    jacobi_eigh(M, B, ev, y);
    // U: r leading even singular vectors on the reduced index, u_s(m) = y_s(m) / sqrt(c_m)
    U.resize((size_t)r * M);
    for (int s = 0; s < r; ++s)
      for (int m = 0; m < M; ++m) U[(size_t)s * M + m] = y[(size_t)m * M + s] / std::sqrt(cm[m]);
    // core: contract m1, then m2, then m3 (weights c_m carry the multiplicities)
    T1.assign((size_t)r * M * M, 0.0);
    for (int a = 0; a < r; ++a)
      for (int m1 = 0; m1 < M; ++m1) {
        const double u = cm[m1] * U[(size_t)a * M + m1];
        const double *h = &H[(size_t)m1 * M * M];
        double *t1 = &T1[(size_t)a * M * M];
        for (size_t i = 0; i < (size_t)M * M; ++i) t1[i] += u * h[i];
      }
    T2.assign((size_t)r * r * M, 0.0);
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b)
        for (int m2 = 0; m2 < M; ++m2) {
          const double u = cm[m2] * U[(size_t)b * M + m2];
          const double *t1 = &T1[((size_t)a * M + m2) * M];
          double *t2 = &T2[((size_t)a * r + b) * M];
          for (int m3 = 0; m3 < M; ++m3) t2[m3] += u * t1[m3];
        }
    beta.assign((size_t)r * r * r, 0.0);
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b)
        for (int c = 0; c < r; ++c) {
          double s = 0.0;
          for (int m3 = 0; m3 < M; ++m3) s += cm[m3] * U[(size_t)c * M + m3] * T2[((size_t)a * r + b) * M + m3];
          beta[((size_t)a * r + b) * r + c] = s;
        }
    // Tucker-to-canonical: eigenpairs of the symmetric mode-3 slices
    std::vector<std::vector<double>> sw(r), sv(r);
    double smax = 0.0;
    for (int c = 0; c < r; ++c) {
      std::vector<double> S((size_t)r * r);
      for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b)
          S[(size_t)a * r + b] = 0.5 * (beta[((size_t)a * r + b) * r + c] + beta[((size_t)b * r + a) * r + c]);
      jacobi_eigh(r, S, sw[c], sv[c]);
      for (int s = 0; s < r; ++s) smax = std::max(smax, std::fabs(sw[c][s]));
    }
    std::vector<double> t1s, t2s, t3s;  // term factors on the reduced index
    int R = 0;
    for (int c = 0; c < r; ++c)
      for (int s = 0; s < r; ++s) {
        if (tol > 0.0 && !(std::fabs(sw[c][s]) > tol * smax)) continue;
        for (int m = 0; m < M; ++m) {
          double v = 0.0;
          for (int a = 0; a < r; ++a) v += U[(size_t)a * M + m] * sv[c][(size_t)a * r + s];
          t1s.push_back(sw[c][s] * v);
          t2s.push_back(v);
          t3s.push_back(U[(size_t)c * M + m]);
        }
        ++R;
      }
    if (R < 1 || R > kMaxRank) return SQ_EINVAL;
    f.assign((size_t)3 * R * N, 0.0);
    const std::vector<double> *ts[3] = {&t1s, &t2s, &t3s};
    for (int ax = 0; ax < 3; ++ax)
      for (int q = 0; q < R; ++q)
        for (int k = 0; k < N; ++k) f[((size_t)ax * R + q) * N + k] = (*ts[ax])[(size_t)q * M + std::min(k, N - k)];
    return precond_create(N, R, f.data(), {}, {}, out);
  } catch (...) {
    return SQ_ENOMEM;
  }
}

}  // extern "C"
