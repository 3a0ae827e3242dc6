// Allocation-free forward transform (ash_forward_noalloc, see include/ash.h).
//
// Who needs it: callers that may not allocate device memory themselves --
// code running inside a host framework that owns every byte of device memory
// and forbids cudaMalloc once it has started, real-time SLM control loops
// that must not allocate while running, and plugins that are only ever
// handed pre-allocated buffers. Such callers cannot create a handle (which
// allocates its workspace), so this entry point takes the basis and all
// other inputs directly as caller buffers.
//
// The forward needs scratch for its split-M partial sums. Here that scratch
// is a file-scope __device__ array of fixed size: it is part of the loaded
// module, so every GPU that loads the library holds it until the process
// exits, and no call allocates anything.
#include <mutex>

#include "ash.h"
#include "transform_kernels.cuh"

namespace ash {
void record_error(const char* msg);
}

namespace {

using namespace ash;

// 2 Mi floats = 8 MiB of split-M partial sums.
constexpr size_t kNoallocScratchFloats = size_t(2) << 20;
static __device__ __align__(256) float g_noalloc_scratch[kNoallocScratchFloats];

// Largest N accepted: one CTA row block (up to 8 warps) must fit the scratch.
constexpr int kNoallocMaxSpots = 131072;
constexpr int kMaxDevices = 64;

struct DirectParams {
  int nx, ny, tiles_x, T, N;
  const float* basis;   // caller basis [D][ny][nx]
  const float* amp;     // [ny][nx]
  const float* phase;   // [ny][nx]
  const float* coeff;   // [N][D]
  float* partial;       // scratch [rows][2N]
  int tiles_per_cta;
};

// Same arithmetic as k_forward, with the basis read from the caller's
// row-major planes and the anchor subtraction done in the kernel (the fp32
// difference of two fp32 values is the correctly rounded exact difference,
// as in the handle's set-up kernel).
template <int D, int P>
__global__ void __launch_bounds__(kTilePix / P) k_forward_noalloc(const DirectParams p) {
  constexpr int NT = kTilePix / P;
  constexpr int NW = NT / 32;
  constexpr int RS = NT / 32;
  constexpr int CPS = cpair_stride(D);
  constexpr float kInv2PiHi = 0.15915494f;
  constexpr float kInv2PiLo = 6.4206382e-09f;   // 1/(2 pi) - kInv2PiHi
  extern __shared__ float4 smem4[];
  float* sC = reinterpret_cast<float*>(smem4);
  float2* sRot = reinterpret_cast<float2*>(sC + kSpotChunk * CPS);

  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int N = p.N;
  const size_t M = (size_t)p.nx * p.ny;
  float* prow = p.partial + (size_t)(blockIdx.x * NW + w) * 2 * N;

  for (int it = 0; it < p.tiles_per_cta; ++it) {
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= p.T) break;
    const bool first = (it == 0);
    const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
    const int x0 = tx * kTileX, y0 = ty * kTileY;
    const int ia = (x0 + min(x0 + kTileX, p.nx) - 1) / 2;
    const int ja = (y0 + min(y0 + kTileY, p.ny) - 1) / 2;
    const size_t ma = (size_t)ja * p.nx + ia;
    float za[D];
    float2 anc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      za[d] = __ldg(p.basis + d * M + ma);
      const float hi = za[d] * kInv2PiHi;
      const float lo = fmaf(za[d], kInv2PiHi, -hi) + za[d] * kInv2PiLo;
      anc[d] = make_float2(hi, lo);
    }

    const int i = x0 + lane;
    float2 dz[P / 2][D];
    float fr[P], fi[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int j = y0 + w + RS * k;
      const bool valid = (i < p.nx) && (j < p.ny);
      const size_t m = (size_t)j * p.nx + i;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float v = valid ? __fsub_rn(__ldg(p.basis + d * M + m), za[d]) : 0.0f;
        if (k & 1) dz[k >> 1][d].y = v;
        else dz[k >> 1][d].x = v;
      }
      float s = 0.0f, c = 0.0f, a = 0.0f;
      if (valid) {
        a = __ldg(p.amp + m);
        sincosf(__ldg(p.phase + m), &s, &c);
      }
      fr[k] = a * c;
      fi[k] = a * s;
    }
    float2 fr2[P / 2], fi2[P / 2], nfr2[P / 2];
#pragma unroll
    for (int q = 0; q < P / 2; ++q) {
      fr2[q] = make_float2(fr[2 * q], fr[2 * q + 1]);
      fi2[q] = make_float2(fi[2 * q], fi[2 * q + 1]);
      nfr2[q] = make_float2(-fr[2 * q], -fr[2 * q + 1]);
    }

    for (int n0 = 0; n0 < N; n0 += kSpotChunk) {
      const int nc = min(kSpotChunk, N - n0);
      __syncthreads();
      for (int s = t; s < nc; s += NT) {
        float c[D];
        float* row = sC + s * CPS;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          c[d] = __ldg(p.coeff + (size_t)(n0 + s) * D + d);
          row[2 * d] = c[d];
          row[2 * d + 1] = c[d];
        }
        sRot[s] = cis_turns(-base_turns<D>(c, anc));
      }
      __syncthreads();

      for (int b0 = 0; b0 < nc; b0 += kBatch) {
        float acc[32];
#pragma unroll
        for (int s = 0; s < kBatch; ++s) {
          float re = 0.0f, im = 0.0f;
          if (b0 + s < nc) {
            float2 cc[D];
            load_cpairs<D>(sC + (b0 + s) * CPS, cc);
            float2 re2 = make_float2(0.0f, 0.0f), im2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int q = 0; q < P / 2; ++q) {
              const float2 x = local_phase<D>(cc, dz[q]);
              float2 sn, cs;
              sincos2(x, sn, cs);
              re2 = fma2(fr2[q], cs, re2);
              re2 = fma2(fi2[q], sn, re2);
              im2 = fma2(fi2[q], cs, im2);
              im2 = fma2(nfr2[q], sn, im2);
            }
            re = re2.x + re2.y;
            im = im2.x + im2.y;
          }
          acc[2 * s] = re;
          acc[2 * s + 1] = im;
        }
        const float v = warp_transpose_reduce32(acc, lane);
        const float other = __shfl_xor_sync(kFull, v, 1);
        const int s = lane >> 1;
        const bool is_im = (lane & 1) != 0;
        if (b0 + s < nc) {
          const float re = is_im ? other : v;
          const float im = is_im ? v : other;
          const float2 r = sRot[b0 + s];
          const float out = is_im ? fmaf(im, r.x, re * r.y) : fmaf(re, r.x, -im * r.y);
          float* dst = prow + 2 * (n0 + b0) + lane;
          *dst = first ? out : (*dst + out);
        }
      }
    }
  }
}

// out[c] = sum over rows of in[r][c], rows in a fixed order.
__global__ void k_noalloc_reduce(const float* __restrict__ in, int rows, int cols, float* __restrict__ out) {
  __shared__ float red[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.0f;
  if (c < cols) {
    for (int r = threadIdx.y; r < rows; r += 32) s += in[(size_t)r * cols + c];
  }
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  for (int h = 16; h >= 1; h >>= 1) {
    if (threadIdx.y < h) red[threadIdx.y][threadIdx.x] += red[threadIdx.y + h][threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.y == 0 && c < cols) out[c] = red[0][threadIdx.x];
}

struct DeviceSetup {
  bool ready = false;
  float* scratch = nullptr;   // device address of g_noalloc_scratch
  int sms = 0;
  int per_sm[ASH_MAX_MODES + 1] = {};   // resident CTAs per SM of the kernel for D modes
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Resident CTAs per SM of the kernel for D modes (part of the one-time
// set-up per device, so that a call does no occupancy query).
template <int D>
cudaError_t occupancy_of(int* out) {
  constexpr int P = pixels_per_thread(D);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_forward_noalloc<D, P>, kTilePix / P,
                                                       fwd_smem_bytes(D));
}

template <int LO, int HI>
cudaError_t fill_occupancy(int* per_sm) {
  if constexpr (LO > HI) {
    return cudaSuccess;
  } else {
    cudaError_t e = occupancy_of<LO>(&per_sm[LO]);
    if (e != cudaSuccess) return e;
    return fill_occupancy<LO + 1, HI>(per_sm);
  }
}

template <int D>
cudaError_t launch_direct(const DirectParams& base, const DeviceSetup& ds, float* E, cudaStream_t s) {
  constexpr int P = pixels_per_thread(D);
  constexpr int NT = kTilePix / P;
  constexpr int NW = NT / 32;
  const int per_sm = ds.per_sm[D];
  cudaError_t e = cudaSuccess;
  const long long cap_rows = (long long)(kNoallocScratchFloats / (2 * (size_t)base.N));
  long long grid = (long long)ds.sms * (per_sm > 0 ? per_sm : 1);
  if (grid > base.T) grid = base.T;
  if (grid * NW > cap_rows) grid = cap_rows / NW;
  if (grid < 1) return cudaErrorInvalidValue;
  DirectParams p = base;
  p.partial = ds.scratch;
  p.tiles_per_cta = (int)((p.T + grid - 1) / grid);
  k_forward_noalloc<D, P><<<(int)grid, NT, fwd_smem_bytes(D), s>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int cols = 2 * p.N;
  k_noalloc_reduce<<<(cols + 31) / 32, dim3(32, 32), 0, s>>>(ds.scratch, (int)grid * NW, cols, E);
  return cudaGetLastError();
}

template <int LO, int HI>
cudaError_t dispatch_direct(int D, const DirectParams& p, const DeviceSetup& ds, float* E, cudaStream_t s) {
  if constexpr (LO > HI) {
    return cudaErrorInvalidValue;
  } else {
    return D == LO ? launch_direct<LO>(p, ds, E, s) : dispatch_direct<LO + 1, HI>(D, p, ds, E, s);
  }
}

ash_status fail(ash_status st, const char* msg) {
  ash::record_error(msg);
  return st;
}

}  // namespace

extern "C" ash_status ash_forward_noalloc(int nx, int ny, const float* amp, const float* phase, int D,
                                         const float* basis, int N, const float* coeff, float* E, void* stream) {
  if (nx < 1 || ny < 1 || nx > 16384 || ny > 16384) return fail(ASH_ERR_INVALID_ARG, "noalloc: grid outside [1, 16384]");
  if (D < 1 || D > ASH_MAX_MODES) return fail(ASH_ERR_INVALID_ARG, "noalloc: D outside [1, ASH_MAX_MODES]");
  if (N < 1 || N > kNoallocMaxSpots)
    return fail(ASH_ERR_INVALID_ARG, "noalloc: N outside [1, 131072] (the fixed 8 MiB scratch holds the "
                                     "partial sums of at most 131072 spots)");
  if (!amp || !phase || !basis || !coeff || !E) return fail(ASH_ERR_INVALID_ARG, "noalloc: NULL buffer");
  if (reinterpret_cast<uintptr_t>(E) & 7) return fail(ASH_ERR_INVALID_ARG, "noalloc: E must be 8-byte aligned");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(ASH_ERR_CUDA, "noalloc: no current CUDA device");
  }
  DeviceSetup ds;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup& slot = g_setup[dev];
    if (!slot.ready) {
      // One-time set-up per device, with that device current: the host-side
      // name g_noalloc_scratch is not a device address; ask the runtime for it.
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || ptr == nullptr) {
        cudaGetLastError();
        return fail(ASH_ERR_CUDA, "noalloc: cudaGetSymbolAddress of the scratch array failed");
      }
      e = cudaDeviceGetAttribute(&slot.sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ASH_ERR_CUDA, "noalloc: cudaDeviceGetAttribute failed");
      }
      e = fill_occupancy<1, ASH_MAX_MODES>(slot.per_sm);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ASH_ERR_CUDA, "noalloc: occupancy query failed");
      }
      slot.scratch = static_cast<float*>(ptr);
      slot.ready = true;
    }
    ds = slot;
  }
  DirectParams p{};
  p.nx = nx;
  p.ny = ny;
  p.tiles_x = (nx + kTileX - 1) / kTileX;
  p.T = p.tiles_x * ((ny + kTileY - 1) / kTileY);
  p.N = N;
  p.basis = basis;
  p.amp = amp;
  p.phase = phase;
  p.coeff = coeff;
  cudaError_t e = dispatch_direct<1, ASH_MAX_MODES>(D, p, ds, E, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(ASH_ERR_CUDA, cudaGetErrorString(e));
  return ASH_OK;
}
