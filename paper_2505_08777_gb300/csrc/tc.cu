// Launchers of the tensor-core transform path (one instantiation per number
// of K-atoms, NA = 1 for D <= 10 and NA = 2 for D <= 21).
#include "tc_kernels.cuh"

namespace ash {

// Resident CTAs per SM from the kernel's registers, shared memory and TMEM
// columns (the runtime's occupancy query does not account for TMEM).
cudaError_t tc_ctas_per_sm(const void* fn, size_t smem, int tmem_cols, int* out) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int warps = kTcThreads / 32;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
  const int by_regs = regs_sm / (regs_warp * warps);
  const int by_smem = (int)((size_t)smem_sm / (smem + fa.sharedSizeBytes + (size_t)reserved));
  const int by_tmem = 512 / tmem_cols;
  int n = by_regs < by_smem ? by_regs : by_smem;
  n = n < by_tmem ? n : by_tmem;
  *out = n < 1 ? 1 : n;
  return cudaSuccess;
}

namespace {

template <int NA>
cudaError_t prepare_na(int* adj, int* fwd) {
  const void* ka = (const void*)k_tc_adjoint<NA>;
  const void* kf = (const void*)k_tc_forward<NA>;
  cudaError_t e;
  // the batched kernels share the single-hologram kernels' shapes
  for (const void* k : {(const void*)k_tc_adjoint_batch<NA>, (const void*)k_tc_forward_batch<NA>}) {
    const int smem = k == (const void*)k_tc_adjoint_batch<NA> ? (int)TcAdjShape<NA>::SMEM : (int)TcFwdShape<NA>::SMEM;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)))
      return e;
  }
  for (const void* k : {ka, (const void*)k_tc_adjoint<NA, false>}) {
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcAdjShape<NA>::SMEM)))
      return e;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)))
      return e;
  }
  if ((e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcFwdShape<NA>::SMEM)))
    return e;
  if ((e = cudaFuncSetAttribute(kf, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared)))
    return e;
  if ((e = tc_ctas_per_sm(ka, TcAdjShape<NA>::SMEM, 2 * kTcChunk, adj))) return e;
  // the gradient's instantiation must fit the same grid
  int adj_grad = 0;
  if ((e = tc_ctas_per_sm((const void*)k_tc_adjoint<NA, false>, TcAdjShape<NA>::SMEM, 2 * kTcChunk, &adj_grad)))
    return e;
  if (adj_grad < *adj) *adj = adj_grad;
  return tc_ctas_per_sm(kf, TcFwdShape<NA>::SMEM, 2 * kTcChunk, fwd);
}

unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// The small kernels that run between the tensor-core launches ask for the
// same shared-memory carveout as those, so that no SM has to change its
// L1 / shared split when the next tensor-core kernel starts. (Measured: with
// their default carveout, a forward with a replicated partial spot block ran
// at 253, 271 or 290 us at 1024^2, N = 400, depending on the kernels before
// it; with it, 252-254 us after every preceding sequence but another
// forward.)
cudaError_t tc_small_kernels_max_shared() {
  cudaError_t e = cudaSuccess;
  for (const void* k : {(const void*)k_tc_field_img, (const void*)k_tc_forward_reduce,
                        (const void*)k_tc_adjoint_fixup, (const void*)k_tc_field_img_batch,
                        (const void*)k_tc_forward_reduce_batch, (const void*)k_tc_adjoint_fixup_batch})
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)))
      return e;
  return e;
}

cudaError_t tc_prepare(int NA, int* adj_ctas_per_sm, int* fwd_ctas_per_sm) {
  cudaError_t e0 = tc_small_kernels_max_shared();
  if (e0 != cudaSuccess) return e0;
  if (NA == 1) return prepare_na<1>(adj_ctas_per_sm, fwd_ctas_per_sm);
  if (NA == 2) return prepare_na<2>(adj_ctas_per_sm, fwd_ctas_per_sm);
  return cudaErrorInvalidValue;
}

cudaError_t tc_batch_ctas_per_sm(int NA, int* adj, int* fwd) {
  cudaError_t e;
  if (NA == 1) {
    if ((e = tc_ctas_per_sm((const void*)k_tc_adjoint_batch<1>, TcAdjShape<1>::SMEM, 2 * kTcChunk, adj))) return e;
    return tc_ctas_per_sm((const void*)k_tc_forward_batch<1>, TcFwdShape<1>::SMEM, 2 * kTcChunk, fwd);
  }
  if (NA == 2) {
    if ((e = tc_ctas_per_sm((const void*)k_tc_adjoint_batch<2>, TcAdjShape<2>::SMEM, 2 * kTcChunk, adj))) return e;
    return tc_ctas_per_sm((const void*)k_tc_forward_batch<2>, TcFwdShape<2>::SMEM, 2 * kTcChunk, fwd);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tc_launch_adjoint(int NA, const TcAdjParams& p, int grid, cudaStream_t s) {
  const bool grad = (p.out.epilogue & kEpiGradPhase) != 0;   // a gradient's single pass: MUFU unreduced
  if (NA == 1 && !grad) k_tc_adjoint<1><<<grid, kTcThreads, TcAdjShape<1>::SMEM, s>>>(p);
  else if (NA == 1) k_tc_adjoint<1, false><<<grid, kTcThreads, TcAdjShape<1>::SMEM, s>>>(p);
  else if (NA == 2 && !grad) k_tc_adjoint<2><<<grid, kTcThreads, TcAdjShape<2>::SMEM, s>>>(p);
  else if (NA == 2) k_tc_adjoint<2, false><<<grid, kTcThreads, TcAdjShape<2>::SMEM, s>>>(p);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t tc_launch_adjoint_batch(int NA, const TcAdjParams* ps, const TcBatchSched& bs, cudaStream_t s) {
  if (NA == 1) k_tc_adjoint_batch<1><<<bs.G, kTcThreads, TcAdjShape<1>::SMEM, s>>>(ps, bs);
  else if (NA == 2) k_tc_adjoint_batch<2><<<bs.G, kTcThreads, TcAdjShape<2>::SMEM, s>>>(ps, bs);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t tc_launch_adjoint_fixup_batch(const TcAdjParams* ps, const int4* list, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_tc_adjoint_fixup_batch<<<n, kTcThreads, 0, s>>>(ps, list);
  return cudaGetLastError();
}

cudaError_t tc_launch_forward_batch(int NA, const TcFwdParams* ps, const TcBatchSched& bs, cudaStream_t s) {
  if (NA == 1) k_tc_forward_batch<1><<<bs.G, kTcThreads, TcFwdShape<1>::SMEM, s>>>(ps, bs);
  else if (NA == 2) k_tc_forward_batch<2><<<bs.G, kTcThreads, TcFwdShape<2>::SMEM, s>>>(ps, bs);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t tc_launch_forward_reduce_batch(const TcFwdParams* ps, const int4* list, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_tc_forward_reduce_batch<<<dim3(n, kTcRows / 32), dim3(32, 32), 0, s>>>(ps, list);
  return cudaGetLastError();
}

cudaError_t tc_field_img_batch(const TcFieldDesc* ds, const int* tiles0, int count, int total_tiles, cudaStream_t s) {
  const long long px = (long long)total_tiles * kTilePix;
  k_tc_field_img_batch<<<blocks_for(px, 256), 256, 0, s>>>(ds, tiles0, count, total_tiles);
  return cudaGetLastError();
}

cudaError_t tc_launch_adjoint_fixup(const TcAdjParams& p, int n_split_groups, cudaStream_t s) {
  if (n_split_groups <= 0) return cudaSuccess;
  k_tc_adjoint_fixup<<<n_split_groups, kTcThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t tc_launch_forward(int NA, const TcFwdParams& p, int grid, cudaStream_t s) {
  if (NA == 1) k_tc_forward<1><<<grid, kTcThreads, TcFwdShape<1>::SMEM, s>>>(p);
  else if (NA == 2) k_tc_forward<2><<<grid, kTcThreads, TcFwdShape<2>::SMEM, s>>>(p);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t tc_launch_forward_reduce(const TcFwdParams& p, cudaStream_t s) {
  k_tc_forward_reduce<<<dim3(p.sched.nb, kTcRows / 32), dim3(32, 32), 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t tc_build_zs(const Geometry& g, const TcLayout& L, const float* dz, float* zs, cudaStream_t s) {
  const long long rows = (long long)g.T * kTcChunksPerTile * kTcChunk;
  k_tc_build_zs<<<blocks_for(rows, 256), 256, 0, s>>>(g, L, dz, zs);
  return cudaGetLastError();
}

cudaError_t tc_build_coeff(const Geometry& g, const TcLayout& L, const float* coeff, const float2* anchors, float* czs,
                           float2* rot, cudaStream_t s) {
  const int nc64 = tc_spot_chunks(g.N);
  k_tc_build_czs<<<blocks_for((long long)(nc64 + 2) * kTcChunk, 256), 256, 0, s>>>(coeff, g.N, L, nc64,
                                                                                 tc_fwd_rep(g.N), czs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long nr = (long long)g.N * g.T;
  k_tile_rotations<<<blocks_for(nr, 256), 256, 0, s>>>(coeff, anchors, g.N, g.D, g.T, rot);
  return cudaGetLastError();
}

cudaError_t tc_field_img(const Geometry& g, const float* amp_img, const float* phase, const float2* field,
                         float4* fimg, cudaStream_t s) {
  const long long px = (long long)g.T * kTilePix;
  k_tc_field_img<<<blocks_for(px, 256), 256, 0, s>>>(g, amp_img, phase, field, reinterpret_cast<float*>(fimg));
  return cudaGetLastError();
}

}  // namespace ash
