// Instantiation helper: defines the launchers of one D range.
#pragma once

#include "launch.h"
#include "transform_kernels.cuh"

namespace ash {

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
    return e;
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
  }
