// Principal isoplanatic modes (paper, Methods "Anisoplanatic Singular Value
// Decomposition"; Sec. III): the SVD W = U Sigma V^T of the N x P block of
// the coefficient matrix formed by the chosen modes rotates those P Zernike
// modes into P principal modes, ordered by singular value; keeping the K
// largest gives the truncated correction Sigma_K. Since
//   sum_d W_nd Z_d = sum_k (U Sigma)_nk (V^T Z)_k,
// the rotated problem has coefficients U Sigma and basis rows V^T Z, and the
// transform kernels run unchanged with D -> D - P + K.
//
// Host code, fp64: one-sided (Hestenes) Jacobi, which orthogonalises the
// columns of W V by plane rotations until every pair is orthogonal; then
// sigma_k = |column k| and the columns themselves are (U Sigma)_k.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ash.h"

namespace ash {
ash_status status_invalid(const char* msg);
}

namespace {

// Columns of A (n x p, column-major) orthogonalised in place; V (p x p,
// column-major) accumulates the rotations.
void jacobi_svd(int n, int p, std::vector<double>& A, std::vector<double>& V) {
  V.assign((size_t)p * p, 0.0);
  for (int k = 0; k < p; ++k) V[(size_t)k * p + k] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int a = 0; a < p - 1; ++a)
      for (int b = a + 1; b < p; ++b) {
        double* x = &A[(size_t)a * n];
        double* y = &A[(size_t)b * n];
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < n; ++i) {
          alpha += x[i] * x[i];
          beta += y[i] * y[i];
          gamma += x[i] * y[i];
        }
        if (gamma == 0.0 || std::fabs(gamma) <= 1e-15 * std::sqrt(alpha * beta)) continue;
        off = std::max(off, std::fabs(gamma) / std::sqrt(alpha * beta));
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < n; ++i) {
          const double xi = x[i], yi = y[i];
          x[i] = c * xi - s * yi;
          y[i] = s * xi + c * yi;
        }
        double* va = &V[(size_t)a * p];
        double* vb = &V[(size_t)b * p];
        for (int i = 0; i < p; ++i) {
          const double xi = va[i], yi = vb[i];
          va[i] = c * xi - s * yi;
          vb[i] = s * xi + c * yi;
        }
      }
    if (off <= 1e-15) break;
  }
}

}  // namespace

extern "C" ash_status ash_principal_modes(int N, int D, const float* coeff, int ncols, const int* cols, int K,
                                          double* mix, float* coeff_out, double* sigma) {
  if (N < 1 || D < 1 || D > ASH_MAX_MODES || !coeff || !cols || !mix || !coeff_out)
    return ash::status_invalid("ash_principal_modes: bad sizes or NULL pointer");
  if (ncols < 1 || ncols > D || K < 0 || K > ncols)
    return ash::status_invalid("ash_principal_modes: need 1 <= ncols <= D and 0 <= K <= ncols");
  std::vector<int> in_cols(D, 0);
  for (int j = 0; j < ncols; ++j) {
    if (cols[j] < 0 || cols[j] >= D || in_cols[cols[j]])
      return ash::status_invalid("ash_principal_modes: cols must be distinct mode positions in [0, D)");
    in_cols[cols[j]] = 1;
  }
  const int P = ncols, Dout = D - P + K;
  std::vector<double> A((size_t)N * P), V;
  for (int j = 0; j < P; ++j)
    for (int n = 0; n < N; ++n) A[(size_t)j * N + n] = (double)coeff[(size_t)n * D + cols[j]];
  jacobi_svd(N, P, A, V);
  // order by singular value; sign fixed so that the largest |entry| of each
  // rotation column is positive (the decomposition is unique up to sign)
  std::vector<double> sv(P);
  std::vector<int> order(P);
  for (int k = 0; k < P; ++k) {
    double s2 = 0.0;
    for (int n = 0; n < N; ++n) s2 += A[(size_t)k * N + n] * A[(size_t)k * N + n];
    sv[k] = std::sqrt(s2);
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sv[a] > sv[b]; });
  if (sigma)
    for (int k = 0; k < P; ++k) sigma[k] = sv[order[k]];
  std::memset(mix, 0, sizeof(double) * (size_t)Dout * D);
  int row = 0;
  for (int d = 0; d < D; ++d) {   // untouched modes first, in order
    if (in_cols[d]) continue;
    mix[(size_t)row * D + d] = 1.0;
    for (int n = 0; n < N; ++n) coeff_out[(size_t)n * Dout + row] = coeff[(size_t)n * D + d];
    ++row;
  }
  for (int k = 0; k < K; ++k, ++row) {
    const int src = order[k];
    const double* v = &V[(size_t)src * P];
    int big = 0;
    for (int j = 1; j < P; ++j)
      if (std::fabs(v[j]) > std::fabs(v[big])) big = j;
    const double sgn = v[big] < 0 ? -1.0 : 1.0;
    for (int j = 0; j < P; ++j) mix[(size_t)row * D + cols[j]] = sgn * v[j];
    for (int n = 0; n < N; ++n) coeff_out[(size_t)n * Dout + row] = (float)(sgn * A[(size_t)src * N + n]);
  }
  return ASH_OK;
}
