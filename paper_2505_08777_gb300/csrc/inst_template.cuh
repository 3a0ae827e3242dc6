// Instantiation helper: defines the launchers of one D range.
#pragma once

#include "launch.h"
#include "tc_kernels.cuh"
#include "transform_kernels.cuh"

namespace ash {

// Resident CTAs per SM from the kernel's registers, shared memory and TMEM
// columns (the runtime's occupancy query is not used for kernels that
// allocate tensor memory).
inline cudaError_t tc_ctas_per_sm(const void* fn, int threads, size_t smem, int tmem_cols, int* out) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
  int by_regs = regs_sm / (regs_warp * warps);
  int by_smem = (int)((size_t)smem_sm / (smem + fa.sharedSizeBytes + (size_t)reserved));
  int by_tmem = 512 / tmem_cols;
  int n = by_regs < by_smem ? by_regs : by_smem;
  n = n < by_tmem ? n : by_tmem;
  *out = n < 1 ? 1 : n;
  return cudaSuccess;
}

template <int D>
struct Inst {
  static constexpr int P = pixels_per_thread(D);
  static constexpr int NT = kTilePix / P;

  static cudaError_t prepare(LaunchInfo* info) {
    cudaError_t e;
    e = cudaFuncSetAttribute(k_forward<D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem_bytes(D));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_adjoint<D, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_smem_bytes(D));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gradc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gradc_smem_bytes(D));
    if (e != cudaSuccess) return e;
    info->threads = NT;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&info->fwd_ctas_per_sm, k_forward<D, P>, NT, fwd_smem_bytes(D));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&info->adj_ctas_per_sm, k_adjoint<D, P>, NT, adj_smem_bytes(D));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&info->gradc_ctas_per_sm, k_gradc<D>, kGradThreads,
                                                      gradc_smem_bytes(D));
    if (e != cudaSuccess) return e;
    info->tc_adj_ctas_per_sm = 0;
    if constexpr (D <= 12) {
      e = cudaFuncSetAttribute(k_tc_adjoint<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(D));
      if (e != cudaSuccess) return e;
      // three ~70 KB CTAs per SM need the largest shared-memory carveout
      e = cudaFuncSetAttribute(k_tc_adjoint<D>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      e = tc_ctas_per_sm((const void*)k_tc_adjoint<D>, kTcThreads, tc_smem_bytes(D), 2 * tc_mb(D) * kTcS,
                         &info->tc_adj_ctas_per_sm);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k_tc_forward<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(D));
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k_tc_forward<D>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      e = tc_ctas_per_sm((const void*)k_tc_forward<D>, kTcThreads, tc_smem_bytes(D), 2 * tc_mb(D) * kTcS,
                         &info->tc_fwd_ctas_per_sm);
    } else {
      info->tc_fwd_ctas_per_sm = 0;
    }
    return e;
  }
  static cudaError_t tc_forward(const TcFwdParams& p, int grid, cudaStream_t s) {
    if constexpr (D <= 12) {
      k_tc_forward<D><<<grid, kTcThreads, tc_smem_bytes(D), s>>>(p);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  static cudaError_t tc_adjoint(const TcAdjParams& p, int grid, cudaStream_t s) {
    if constexpr (D <= 12) {
      k_tc_adjoint<D><<<grid, kTcThreads, tc_smem_bytes(D), s>>>(p);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  static cudaError_t forward(const FwdParams& p, int grid, cudaStream_t s) {
    k_forward<D, P><<<grid, NT, fwd_smem_bytes(D), s>>>(p);
    return cudaGetLastError();
  }
  static cudaError_t adjoint(const AdjParams& p, int grid, cudaStream_t s) {
    k_adjoint<D, P><<<grid, NT, adj_smem_bytes(D), s>>>(p);
    return cudaGetLastError();
  }
  static cudaError_t gradc(const GradCParams& p, dim3 grid, cudaStream_t s) {
    k_gradc<D><<<grid, kGradThreads, gradc_smem_bytes(D), s>>>(p);
    return cudaGetLastError();
  }
};

template <int LO, int HI>
struct Range {
  static cudaError_t prepare(int D, LaunchInfo* info) {
    if constexpr (LO > HI) return cudaErrorInvalidValue;
    else return D == LO ? Inst<LO>::prepare(info) : Range<LO + 1, HI>::prepare(D, info);
  }
  static cudaError_t forward(int D, const FwdParams& p, int grid, cudaStream_t s) {
    if constexpr (LO > HI) return cudaErrorInvalidValue;
    else return D == LO ? Inst<LO>::forward(p, grid, s) : Range<LO + 1, HI>::forward(D, p, grid, s);
  }
  static cudaError_t adjoint(int D, const AdjParams& p, int grid, cudaStream_t s) {
    if constexpr (LO > HI) return cudaErrorInvalidValue;
    else return D == LO ? Inst<LO>::adjoint(p, grid, s) : Range<LO + 1, HI>::adjoint(D, p, grid, s);
  }
  static cudaError_t gradc(int D, const GradCParams& p, dim3 grid, cudaStream_t s) {
    if constexpr (LO > HI) return cudaErrorInvalidValue;
    else return D == LO ? Inst<LO>::gradc(p, grid, s) : Range<LO + 1, HI>::gradc(D, p, grid, s);
  }
  static cudaError_t tc_forward(int D, const TcFwdParams& p, int grid, cudaStream_t s) {
    if constexpr (LO > HI) return cudaErrorInvalidValue;
    else return D == LO ? Inst<LO>::tc_forward(p, grid, s) : Range<LO + 1, HI>::tc_forward(D, p, grid, s);
  }
  static cudaError_t tc_adjoint(int D, const TcAdjParams& p, int grid, cudaStream_t s) {
    if constexpr (LO > HI) return cudaErrorInvalidValue;
    else return D == LO ? Inst<LO>::tc_adjoint(p, grid, s) : Range<LO + 1, HI>::tc_adjoint(D, p, grid, s);
  }
};

}  // namespace ash

#define ASH_DEFINE_RANGE(R)                                                                          \
  namespace ash {                                                                                    \
  cudaError_t prepare_r##R(int D, LaunchInfo* info) { return Range<4 * R + 1, 4 * R + 4>::prepare(D, info); } \
  cudaError_t launch_forward_r##R(int D, const FwdParams& p, int grid, cudaStream_t s) {            \
    return Range<4 * R + 1, 4 * R + 4>::forward(D, p, grid, s);                                      \
  }                                                                                                  \
  cudaError_t launch_adjoint_r##R(int D, const AdjParams& p, int grid, cudaStream_t s) {            \
    return Range<4 * R + 1, 4 * R + 4>::adjoint(D, p, grid, s);                                      \
  }                                                                                                  \
  cudaError_t launch_gradc_r##R(int D, const GradCParams& p, dim3 grid, cudaStream_t s) {           \
    return Range<4 * R + 1, 4 * R + 4>::gradc(D, p, grid, s);                                        \
  }                                                                                                  \
  cudaError_t launch_tc_adjoint_r##R(int D, const TcAdjParams& p, int grid, cudaStream_t s) {        \
    return Range<4 * R + 1, 4 * R + 4>::tc_adjoint(D, p, grid, s);                                   \
  }                                                                                                  \
  cudaError_t launch_tc_forward_r##R(int D, const TcFwdParams& p, int grid, cudaStream_t s) {        \
    return Range<4 * R + 1, 4 * R + 4>::tc_forward(D, p, grid, s);                                   \
  }                                                                                                  \
  }
