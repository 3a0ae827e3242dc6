// Conjugate-gradient refinement of the SLM phase (paper Methods: precision
// targets such as uniform top hats refined by conjugate-gradient descent
// through the transform's gradients): PR+ nonlinear CG with a one-trial
// quadratic line search, every scalar on the device in fp64, the loop one
// CUDA graph per iteration count (ash_cg_refine in include/ash.h).
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

// fp64 scalars of the iteration in h->cg_scal
enum CgSlot : int { kCgL = 0, kCgS, kCgA0, kCgL1, kCgA, kCgGG, kCgGN, kCgGX, kCgBeta, kCgMax, kCgTheta, kCgRestart,
                    kCgZero, kCgSlotCount };
static_assert(kCgSlotCount == kCgSlots, "scalar slots of the CG workspace");

// Sum of a double over the block (blockDim.x a multiple of 32, <= 1024) in a
// fixed order; the result is valid in every thread.
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += sh[k];
  return t;
}

// Spot-intensity loss from E (fp64): I = |E|^2, mu = mean I, r = I/mu - t,
// L = sum r^2; with gE, its complex gradient gE = 2 G E,
// G = (2/mu) (r - sum_n(r_n I_n / mu) / N).
__global__ void k_cg_loss(const float2* __restrict__ E, const float* __restrict__ t, int N,
                          float2* __restrict__ gE, double* __restrict__ scal, int slot,
                          float* __restrict__ loss_out) {
  __shared__ double sh[32];
  double sI = 0.0;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const double ex = E[n].x, ey = E[n].y;
    sI += ex * ex + ey * ey;
  }
  const double mu = block_sum(sI, sh) / N;
  double sL = 0.0, sX = 0.0;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const double ex = E[n].x, ey = E[n].y, I = ex * ex + ey * ey, r = I / mu - (double)t[n];
    sL += r * r;
    sX += r * I / mu;
  }
  const double L = block_sum(sL, sh), X = block_sum(sX, sh) / N;
  if (gE) {
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
      const double ex = E[n].x, ey = E[n].y, I = ex * ex + ey * ey, r = I / mu - (double)t[n];
      const double G = (2.0 / mu) * (r - X);
      gE[n] = make_float2((float)(2.0 * G * ex), (float)(2.0 * G * ey));
    }
  }
  if (threadIdx.x == 0) {
    scal[slot] = L;
    if (loss_out) *loss_out = (float)L;
  }
}

// Partial reductions over M in a fixed block order: mode 0 sum a b, mode 1
// max |a|.
__global__ void k_cg_reduce(const float* __restrict__ a, const float* __restrict__ b, long long M, int mode,
                            double* __restrict__ part) {
  __shared__ double sh[32];
  double v = 0.0;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x)
    v = mode == 0 ? v + (double)a[m] * (double)b[m] : fmax(v, fabs((double)a[m]));
  if (mode == 0) {
    v = block_sum(v, sh);
  } else {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v = fmax(v, sh[k]);
  }
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void k_cg_finish(const double* __restrict__ part, int nparts, int mode, double* __restrict__ scal,
                            int slot) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) v = mode == 0 ? v + part[k] : fmax(v, part[k]);
  if (mode == 0) {
    v = block_sum(v, sh);
  } else {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v = fmax(v, sh[k]);
  }
  if (threadIdx.x == 0) scal[slot] = v;
}

// The scalar steps of one CG iteration (one thread), in the order of the
// iteration: 0 restart test on s = g.d; 1 trial step a0 = theta / max|d|;
// 2 step a from the quadratic through L, s and L(a0); 3 beta (PR+).
__global__ void k_cg_step(double* scal, int op) {
  double* c = scal;
  if (op == 0) {
    c[kCgRestart] = c[kCgS] >= 0.0 ? 1.0 : 0.0;
    if (c[kCgS] >= 0.0) c[kCgS] = -c[kCgGG];
  } else if (op == 1) {
    c[kCgA0] = c[kCgMax] > 0.0 ? c[kCgTheta] / c[kCgMax] : 0.0;
  } else if (op == 2) {
    const double a0 = c[kCgA0];
    if (a0 > 0.0) {
      const double curv = (c[kCgL1] - c[kCgL] - c[kCgS] * a0) / (a0 * a0);
      c[kCgA] = curv > 0.0 ? -c[kCgS] / (2.0 * curv) : 2.0 * a0;
    } else {
      c[kCgA] = 0.0;
    }
  } else {
    c[kCgBeta] = c[kCgGG] > 0.0 ? fmax(0.0, (c[kCgGN] - c[kCgGX]) / c[kCgGG]) : 0.0;
    c[kCgGG] = c[kCgGN];
  }
}

// out = x + scal[slot] d
__global__ void k_cg_axpy(float* out, const float* x, const float* __restrict__ d, long long M,
                          const double* __restrict__ scal, int slot) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  out[m] = (float)((double)x[m] + scal[slot] * (double)d[m]);
}

// d = -g + scal[slot] d; with `if_restart`, only when the restart flag is set
__global__ void k_cg_dir(float* __restrict__ d, const float* __restrict__ g, long long M,
                         const double* __restrict__ scal, int slot, int if_restart) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M || (if_restart && scal[kCgRestart] == 0.0)) return;
  d[m] = (float)(-(double)g[m] + scal[slot] * (double)d[m]);
}

// The CG loop on the handle's buffers (phase cg_phase, targets cg_t; scalars
// kCgTheta and kCgZero set by the caller): the loss and gradient at the
// start, then `iters` iterations; loss k in cg_loss[k].
ash_status enqueue_cg_body(ash_hologram* h, int iters, cudaStream_t s) {
  const long long M = (long long)h->g.nx * h->g.ny;
  const int N = h->g.N;
  const unsigned vb = (unsigned)((M + 255) / 256);
  float* g[2] = {h->cg_g, h->cg_g + M};
  double* sc = h->cg_scal;
  auto chk = [&](const char* where) -> ash_status {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ASH_OK : cuda_fail(e, where);
  };
  auto dot = [&](const float* a, const float* b, int mode, int slot) {
    k_cg_reduce<<<kCgRedBlocks, 256, 0, s>>>(a, b, M, mode, h->cg_part);
    k_cg_finish<<<1, 512, 0, s>>>(h->cg_part, kCgRedBlocks, mode, sc, slot);
  };
  ash_status st;
  if ((st = forward_enqueue(h, kSrcPhase, h->cg_phase, nullptr, h->E, s)) != ASH_OK) return st;
  k_cg_loss<<<1, 1024, 0, s>>>(h->E, h->cg_t, N, h->y, sc, kCgL, h->cg_loss);
  if ((st = chk("CG loss launch")) != ASH_OK) return st;
  if ((st = adjoint_enqueue(h, h->y, nullptr, nullptr, h->cg_phase, g[0], kEpiGradPhase, s)) != ASH_OK) return st;
  dot(g[0], g[0], 0, kCgGG);
  k_cg_dir<<<vb, 256, 0, s>>>(h->cg_d, g[0], M, sc, kCgZero, 0);   // d = -g
  if ((st = chk("CG start launch")) != ASH_OK) return st;
  int cur = 0;
  for (int k = 0; k < iters; ++k) {
    dot(g[cur], h->cg_d, 0, kCgS);
    k_cg_step<<<1, 1, 0, s>>>(sc, 0);
    k_cg_dir<<<vb, 256, 0, s>>>(h->cg_d, g[cur], M, sc, kCgZero, 1);   // restart: d = -g
    dot(h->cg_d, nullptr, 1, kCgMax);
    k_cg_step<<<1, 1, 0, s>>>(sc, 1);
    k_cg_axpy<<<vb, 256, 0, s>>>(h->cg_trial, h->cg_phase, h->cg_d, M, sc, kCgA0);
    if ((st = chk("CG trial launch")) != ASH_OK) return st;
    if ((st = forward_enqueue(h, kSrcPhase, h->cg_trial, nullptr, h->E, s)) != ASH_OK) return st;
    k_cg_loss<<<1, 1024, 0, s>>>(h->E, h->cg_t, N, nullptr, sc, kCgL1, nullptr);
    k_cg_step<<<1, 1, 0, s>>>(sc, 2);
    k_cg_axpy<<<vb, 256, 0, s>>>(h->cg_phase, h->cg_phase, h->cg_d, M, sc, kCgA);
    if ((st = chk("CG step launch")) != ASH_OK) return st;
    if ((st = forward_enqueue(h, kSrcPhase, h->cg_phase, nullptr, h->E, s)) != ASH_OK) return st;
    k_cg_loss<<<1, 1024, 0, s>>>(h->E, h->cg_t, N, h->y, sc, kCgL, h->cg_loss + k + 1);
    if ((st = chk("CG loss launch")) != ASH_OK) return st;
    if ((st = adjoint_enqueue(h, h->y, nullptr, nullptr, h->cg_phase, g[cur ^ 1], kEpiGradPhase, s)) != ASH_OK)
      return st;
    dot(g[cur ^ 1], g[cur ^ 1], 0, kCgGN);
    dot(g[cur ^ 1], g[cur], 0, kCgGX);
    k_cg_step<<<1, 1, 0, s>>>(sc, 3);
    k_cg_dir<<<vb, 256, 0, s>>>(h->cg_d, g[cur ^ 1], M, sc, kCgBeta, 0);
    if ((st = chk("CG direction launch")) != ASH_OK) return st;
    cur ^= 1;
  }
  return ASH_OK;
}

}  // namespace

extern "C" {

ash_status ash_cg_refine(ash_hologram* h, float* phase, const float* t, int iters, float theta, float* loss_out,
                         void* stream) {
  if (!h || !phase || !t) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (iters < 0 || iters > kCgMaxIters) return set_error(ASH_ERR_INVALID_ARG, "iters outside [0, %d]", kCgMaxIters);
  if (!(theta > 0.0f && theta <= 3.2f)) return set_error(ASH_ERR_INVALID_ARG, "theta outside (0, 3.2]");
  if (consume_injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = as_stream(stream);
  const size_t M = (size_t)h->g.nx * h->g.ny;
  double init[kCgSlots] = {};
  init[kCgTheta] = theta;
  ASH_CUDA(cudaMemcpyAsync(h->cg_phase, phase, M * 4, cudaMemcpyDeviceToDevice, s));
  ASH_CUDA(cudaMemcpyAsync(h->cg_t, t, (size_t)h->g.N * 4, cudaMemcpyDeviceToDevice, s));
  ASH_CUDA(cudaMemcpyAsync(h->cg_scal, init, sizeof init, cudaMemcpyHostToDevice, s));
  if (iters >= 1) {
    cudaGraphExec_t exec = nullptr;
    ash_status st = cached_graph(h, -iters, enqueue_cg_body, iters, &exec);
    if (st != ASH_OK) return st;
    ASH_CUDA(cudaGraphLaunch(exec, s));
  } else {
    ash_status st = enqueue_cg_body(h, 0, s);
    if (st != ASH_OK) return st;
  }
  ASH_CUDA(cudaMemcpyAsync(phase, h->cg_phase, M * 4, cudaMemcpyDeviceToDevice, s));
  if (loss_out) ASH_CUDA(cudaMemcpyAsync(loss_out, h->cg_loss, (size_t)(iters + 1) * 4, cudaMemcpyDeviceToDevice, s));
  return ASH_OK;
}

}  // extern "C"
