// Pipe-rate probe (ash_probe_rates, see include/ash.h).
//
// The transforms' roofline is built from per-SM unit rates: how many sin /
// cos results the MUFU delivers per clock, and how many FP32 lane results
// the FMA pipe delivers per clock (as scalar fma.rn.f32 and as the packed
// fma.rn.f32x2 the kernels use). This probe measures them on the running
// GPU: one CTA of 1024 threads per SM (its dynamic shared memory request
// leaves room for no second CTA), each thread running independent chains
// of one operation, timed by the SM's own cycle counter between two CTA
// barriers. Rates are results per clock per SM, so they do not depend on
// the clock the GPU happens to run at; that clock is estimated separately
// from the cycle count and the launch's CUDA-event time.
#include <algorithm>
#include <vector>

#include "ash.h"
#include "common.cuh"

namespace ash {
void record_error(const char* msg);
}

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 8;
constexpr size_t kProbeSmem = 120 * 1024;   // > half an SM's shared memory: one CTA per SM

enum ProbeOp : int { kOpSinCos = 0, kOpFfma = 1, kOpFfma2 = 2, kOpEx2 = 3, kNumOps = 4 };

__device__ __forceinline__ float p_sin(float x) {
  float y;
  asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float p_cos(float x) {
  float y;
  asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float p_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float p_fma(float a, float b, float c) {
  float y;
  asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
  return y;
}
__device__ __forceinline__ void p_fma2(float& a0, float& a1, float b, float c) {
  asm volatile(
      "{\n\t.reg .b64 ra, rb, rc;\n\t"
      "mov.b64 ra, {%0, %1};\n\t"
      "mov.b64 rb, {%2, %2};\n\t"
      "mov.b64 rc, {%3, %3};\n\t"
      "fma.rn.f32x2 ra, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, ra;\n\t}"
      : "+f"(a0), "+f"(a1)
      : "f"(b), "f"(c));
}

// Each thread: kChains independent chains, `iters` steps. Results per
// thread and step: sin/cos 8 (4 sin, 4 cos), fma 8, fma2 16 (8 instructions
// of two lanes), ex2 8.
template <int OP>
__global__ void __launch_bounds__(kProbeThreads, 1) k_probe(float seed, int iters, long long* cycles, float* sink) {
  extern __shared__ float pad[];
  float a[2 * kChains];
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) a[k] = seed * (float)(threadIdx.x + 1 + 37 * k) * 1e-4f;
  if (threadIdx.x == 0) pad[0] = seed;
  const float b = 0.999f, c = 1e-3f * seed;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if constexpr (OP == kOpSinCos) a[k] = (k & 1) ? p_cos(a[k]) : p_sin(a[k]);
      if constexpr (OP == kOpFfma) a[k] = p_fma(a[k], b, c);
      if constexpr (OP == kOpFfma2) p_fma2(a[2 * k], a[2 * k + 1], b, c);
      if constexpr (OP == kOpEx2) a[k] = p_ex2(a[k]) - 1.0f;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) s += a[k];
  if (s == 1234.5f) sink[blockIdx.x] = s + pad[0];   // keeps the chains live
}

// Results per thread and step of each operation (see k_probe), and the step
// counts (about 2-4 million SM cycles per launch).
constexpr int kResults[kNumOps] = {kChains, kChains, 2 * kChains, kChains};
constexpr int kIters[kNumOps] = {4096, 16384, 8192, 4096};

template <int OP>
cudaError_t run_op(int sms, long long* d_cycles, float* d_sink, cudaStream_t s, double* rate, double* mhz) {
  cudaError_t e = cudaFuncSetAttribute(k_probe<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeSmem);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev0, ev1;
  if ((e = cudaEventCreate(&ev0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&ev1)) != cudaSuccess) {
    cudaEventDestroy(ev0);
    return e;
  }
  std::vector<long long> cyc(sms);
  float ms = 0.0f;
  // one warm-up launch, then the timed one
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    cudaEventRecord(ev0, s);
    k_probe<OP><<<sms, kProbeThreads, kProbeSmem, s>>>(1.0f, kIters[OP], d_cycles, d_sink);
    e = cudaGetLastError();
    cudaEventRecord(ev1, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(cyc.data(), d_cycles, sms * sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (e != cudaSuccess) return e;
  std::sort(cyc.begin(), cyc.end());
  const double med = (double)cyc[sms / 2];
  const double results = (double)kProbeThreads * kIters[OP] * kResults[OP];
  *rate = med > 0 ? results / med : 0.0;
  *mhz = ms > 0 ? (double)cyc[sms - 1] / (ms * 1e3) : 0.0;
  return cudaSuccess;
}

}  // namespace

extern "C" ash_status ash_probe_rates(double* out, void* stream) {
  if (!out) {
    ash::record_error("probe: out is NULL");
    return ASH_ERR_INVALID_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long* d_cycles = nullptr;
  float* d_sink = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&d_cycles, (size_t)sms * sizeof(long long), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_sink, (size_t)sms * sizeof(float), s);
  double rate[kNumOps] = {}, mhz[kNumOps] = {};
  if (e == cudaSuccess) e = run_op<kOpSinCos>(sms, d_cycles, d_sink, s, &rate[0], &mhz[0]);
  if (e == cudaSuccess) e = run_op<kOpFfma>(sms, d_cycles, d_sink, s, &rate[1], &mhz[1]);
  if (e == cudaSuccess) e = run_op<kOpFfma2>(sms, d_cycles, d_sink, s, &rate[2], &mhz[2]);
  if (e == cudaSuccess) e = run_op<kOpEx2>(sms, d_cycles, d_sink, s, &rate[3], &mhz[3]);
  if (d_cycles) cudaFreeAsync(d_cycles, s);
  if (d_sink) cudaFreeAsync(d_sink, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ash::record_error(cudaGetErrorString(e));
    return ASH_ERR_CUDA;
  }
  for (int k = 0; k < kNumOps; ++k) out[k] = rate[k];
  double m = 0.0;
  for (int k = 0; k < kNumOps; ++k) m += mhz[k];
  out[4] = m / kNumOps;
  out[5] = (double)sms;
  return ASH_OK;
}
