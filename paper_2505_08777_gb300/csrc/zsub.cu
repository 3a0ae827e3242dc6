// Simulated Zernike-subtraction calibration (paper Sec. III: a global
// Zernike order superimposed on the SLM with a swept amplitude, a per-spot
// figure of merit, and the per-spot optimum subtracted in aberration space):
// the sweep through a system handle and the per-spot estimate
// (ash_zsub_sweep / ash_zsub_estimate in include/ash.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "ash.h"
#include "handle.h"

using namespace ash;

namespace {

ash_status set_error(ash_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  record_error(buf);
  return s;
}

ash_status cuda_fail(cudaError_t e, const char* where) { return status_cuda(e, where); }

#define ASH_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// coeff = base - delta e_mode for every spot: the system seen through the
// SLM phase phi + delta Z_mode, since exp(i delta Z_d) exp(-i C . Z) =
// exp(-i (C - delta e_d) . Z).
__global__ void k_zsub_shift(const float* __restrict__ base, float* __restrict__ coeff, int N, int D, int mode,
                             float delta) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)N * D) return;
  coeff[i] = base[i] - ((int)(i % D) == mode ? delta : 0.0f);
}

__global__ void k_abs2(const float2* __restrict__ E, float* __restrict__ I, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float2 e = E[n];
  I[n] = e.x * e.x + e.y * e.y;
}

// Least-squares parabola through (delta_k, ln I_k): P = (X^T X)^-1 X^T with
// rows X_k = (1, delta_k, delta_k^2), from the host in fp64.
constexpr int kZsubMaxK = 32;
struct ZsubFit {
  int K;
  double dmin, dmax;
  double P[3][kZsubMaxK];
  double delta[kZsubMaxK];
};

// Per spot (fp64): (a, b, c) = P ln max(I, 1e-37); the vertex -b / (2 c)
// clipped to the sweep range if c < 0, else the offset of the largest sample.
__global__ void k_zsub_estimate(const float* __restrict__ I, int N, const ZsubFit fit,
                                float* __restrict__ out, float* __restrict__ coeff, int D, int mode) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double b = 0.0, c = 0.0, best = -1e300;
  int kbest = 0;
  for (int k = 0; k < fit.K; ++k) {
    const double L = log((double)fmaxf(I[(size_t)k * N + n], 1e-37f));
    b += fit.P[1][k] * L;
    c += fit.P[2][k] * L;
    if (L > best) {
      best = L;
      kbest = k;
    }
  }
  double v = fit.delta[kbest];
  if (c < 0.0) v = fmin(fmax(-b / (2.0 * c), fit.dmin), fit.dmax);
  out[n] = (float)v;
  if (coeff) coeff[(size_t)n * D + mode] += (float)v;
}

}  // namespace

extern "C" {

ash_status ash_zsub_sweep(ash_hologram* h, const float* phase, int mode, const float* deltas, int K, float* intensity,
                          void* stream) {
  if (!h || !phase || !deltas || !intensity) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (mode < 0 || mode >= h->g.D) return set_error(ASH_ERR_INVALID_ARG, "mode %d outside [0, %d)", mode, h->g.D);
  if (K < 1 || K > kZsubMaxK) return set_error(ASH_ERR_INVALID_ARG, "K = %d outside [1, %d]", K, kZsubMaxK);
  if (consume_injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = as_stream(stream);
  const int N = h->g.N, D = h->g.D;
  const size_t bytes = (size_t)N * D * sizeof(float);
  const unsigned blocks = (unsigned)(((size_t)N * D + 255) / 256);
  ASH_CUDA(cudaMemcpyAsync(h->coeff_bak, h->coeff, bytes, cudaMemcpyDeviceToDevice, s));
  ash_status st = ASH_OK;
  for (int k = 0; k < K && st == ASH_OK; ++k) {
    k_zsub_shift<<<blocks, 256, 0, s>>>(h->coeff_bak, h->coeff, N, D, mode, deltas[k]);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = coeff_images_enqueue(h, s);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "calibration sweep");
      break;
    }
    st = forward_enqueue(h, kSrcPhase, phase, nullptr, h->E, s);
    if (st != ASH_OK) break;
    k_abs2<<<(N + 255) / 256, 256, 0, s>>>(h->E, intensity + (size_t)k * N, N);
    if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "calibration sweep");
  }
  // the handle's coefficients and operand images are restored in every case
  cudaError_t e = cudaMemcpyAsync(h->coeff, h->coeff_bak, bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = coeff_images_enqueue(h, s);
  if (st == ASH_OK && e != cudaSuccess) st = cuda_fail(e, "calibration sweep restore");
  return st;
}

ash_status ash_zsub_estimate(const float* intensity, const float* deltas, int K, int N, float* delta_star,
                             float* coeff, int D, int mode, void* stream) {
  if (!intensity || !deltas || !delta_star) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (K < 3 || K > kZsubMaxK) return set_error(ASH_ERR_INVALID_ARG, "K = %d outside [3, %d]", K, kZsubMaxK);
  if (N < 0) return set_error(ASH_ERR_INVALID_ARG, "N < 0");
  if (coeff && (D < 1 || mode < 0 || mode >= D)) return set_error(ASH_ERR_INVALID_ARG, "mode outside [0, D)");
  ZsubFit fit{};
  fit.K = K;
  fit.dmin = fit.dmax = deltas[0];
  double G[3][3] = {};
  for (int k = 0; k < K; ++k) {
    const double d = deltas[k], x[3] = {1.0, d, d * d};
    fit.delta[k] = d;
    fit.dmin = d < fit.dmin ? d : fit.dmin;
    fit.dmax = d > fit.dmax ? d : fit.dmax;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) G[i][j] += x[i] * x[j];
  }
  // (X^T X)^-1 by cofactors; fewer than three distinct offsets make it singular
  const double det = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                     G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                     G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
  const double scale = G[0][0] * G[1][1] * G[2][2];
  if (!(fabs(det) > 1e-12 * scale)) return set_error(ASH_ERR_INVALID_ARG, "need three distinct offsets");
  double Gi[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
      Gi[i][j] = (G[i1][j1] * G[i2][j2] - G[i1][j2] * G[i2][j1]) / det;
    }
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < K; ++k) {
      const double d = deltas[k], x[3] = {1.0, d, d * d};
      fit.P[r][k] = Gi[r][0] * x[0] + Gi[r][1] * x[1] + Gi[r][2] * x[2];
    }
  if (consume_injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  if (N == 0) return ASH_OK;
  k_zsub_estimate<<<(N + 255) / 256, 256, 0, as_stream(stream)>>>(intensity, N, fit, delta_star, coeff, D, mode);
  ASH_CUDA(cudaGetLastError());
  return ASH_OK;
}

}  // extern "C"
