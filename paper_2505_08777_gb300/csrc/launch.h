// Launchers of the D-templated transform kernels (one translation unit per
// range of D so the instantiations compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace ash {

struct LaunchInfo {
  int threads;        // CTA size of the pixel-stationary kernels
  int fwd_ctas_per_sm;
  int adj_ctas_per_sm;
  int gradc_ctas_per_sm;
  int tc_adj_ctas_per_sm;   // 0 if the tensor-core path is not available for this D
  int tc_fwd_ctas_per_sm;
  int tc_grad_ctas_per_sm;   // 0 if the tensor-core moment pass is not available
};

// Each returns cudaErrorInvalidValue when D is outside its range.
#define ASH_DECLARE_RANGE(R)                                                                  \
  cudaError_t prepare_r##R(int D, LaunchInfo* info);                                          \
  cudaError_t launch_forward_r##R(int D, const FwdParams& p, int grid, cudaStream_t s);       \
  cudaError_t launch_adjoint_r##R(int D, const AdjParams& p, int grid, cudaStream_t s);       \
  cudaError_t launch_gradc_r##R(int D, const GradCParams& p, dim3 grid, cudaStream_t s);
ASH_DECLARE_RANGE(0)
ASH_DECLARE_RANGE(1)
ASH_DECLARE_RANGE(2)
ASH_DECLARE_RANGE(3)
#undef ASH_DECLARE_RANGE

// Range r covers D in [4r + 1, 4r + 4].
inline int range_of(int D) { return (D - 1) / 4; }

}  // namespace ash
