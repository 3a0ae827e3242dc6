// Internal definition of the hologram handle (shared by the C-ABI
// translation units; not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <vector>

#include "ash.h"
#include "common.cuh"
#include "launch.h"
#include "mono.h"
#include "tc_launch.h"

struct ash_hologram {
  ash::Geometry g{};
  int device = 0;
  cudaStream_t home = nullptr;     // stream the workspace was allocated on
  ash::LaunchInfo li{};
  ash::Schedule sched{};           // (tile, spot) ranges of the transform kernels
  bool split_tiles = false;   // some tile's spots span two CTA ranges
  int fwd_rows = 0;
  int gradc_gx = 0, gradc_gy = 0;
  // workspace
  float* dz = nullptr;           // register-image basis of the FMA-pipe kernels (NULL while unused)
  int basis_max_order = 0;      // of the monomial tables (rebuilding dz)
  bool user_basis = false;      // created from a caller's basis (dz is never dropped)
  float* amp_img = nullptr;
  float2* anchors = nullptr;
  float* coeff = nullptr;
  float* coeff_bak = nullptr;   // the coefficients during a calibration sweep
  float* partial = nullptr;
  // tensor-core path (D <= 21): operand images, schedules, split buffers
  int variant = 0;              // 0 auto, 1 FMA-pipe kernels, 2 tensor-core kernels
  bool tc_ok = false;
  int tc_na = 0;                // K-atoms per operand row
  ash::TcLayout tc_layout{};
  ash::Schedule tadj{};         // adjoint units (group, spot chunk)
  bool tadj_split = false;      // some group's spots span two CTA ranges
  ash::TcFwdSched tfwd{};       // forward units (spot block, pixel chunk)
  bool tfwd_split = false;      // some spot block's pixels span two CTA ranges
  float* zs = nullptr;
  float* czs = nullptr;
  float4* fimg = nullptr;
  float2* rot = nullptr;        // [T][N] per-(tile, spot) anchor phase rotations
  float2* tc_split = nullptr;   // [tadj.G][2][128]
  float2* tc_part = nullptr;    // [tfwd.G][2][128]
  long long* tfwd_begin = nullptr;   // [tfwd.G + 1] CTA range starts of the forward
  int2* tfwd_spans = nullptr;        // [tfwd.nb] first and last CTA meeting each spot block
  int* tfwd_claim = nullptr;         // [kTcClaimInts] range-claim counters (SM-aware ranges)
  int tfwd_nfull = -1;               // ranges of the full spot blocks, or -1: CTA g runs range g
  long long* tadj_begin = nullptr;   // [tadj.G + 1] CTA range starts of the adjoint
  int4* tadj_groups = nullptr;  // (group, first CTA, last CTA, -) of the groups split between adjoint CTA ranges
  int tadj_nsplit = 0;
  bool tgrad_ok = false;        // tensor-core moment pass of the coefficient gradient (one K-atom)
  ash::TcFwdSched tgrad{};      // its units (spot block, pixel chunk)
  bool tgrad_split = false;     // some spot block's pixels span two CTA ranges
  long long* tgrad_begin = nullptr;  // [tgrad.G + 1]
  int2* tgrad_spans = nullptr;       // [tgrad.nb] first and last CTA meeting each spot block
  float* tgrad_part = nullptr;  // [tgrad.G][2][128][DC]
  int tgrad_ord = 0;            // total degree of the basis polynomials
  float* tpoly = nullptr;       // tile polynomials of the basis
  float2* split = nullptr;
  float* gradc_partial = nullptr;
  float2* E = nullptr;
  float2* y = nullptr;
  float* wgs_phase = nullptr;
  float* wgs_w = nullptr;
  float* wgs_T = nullptr;
  float2* wgs_E = nullptr;
  float2* wgs_u = nullptr;      // spot phases (unit phasors) of the last unfixed update
  float wgs_feedback = 1.0f;    // feedback exponent p of the weight update
  bool wgs_fix = false;         // phase fixing: hold the spot phases at wgs_u
  float* wgs_metrics = nullptr;
  // conjugate-gradient refinement: phase, targets, gradients, direction,
  // trial phase, fp64 scalars, reduction partials, loss history
  float* cg_phase = nullptr;
  float* cg_t = nullptr;
  float* cg_g = nullptr;        // [2][M]
  float* cg_d = nullptr;
  float* cg_trial = nullptr;
  double* cg_scal = nullptr;
  double* cg_part = nullptr;
  float* cg_loss = nullptr;     // [kCgMaxIters + 1]
  double* sum_a2 = nullptr;
  double* sum_a2_arg = nullptr;   // a caller's total sum A^2 (ash_spot_metrics)
  ash::MonoTerm* terms = nullptr;
  int* term_off = nullptr;
  unsigned* err_word = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  cudaStream_t capture = nullptr;
  // WGS loops by iteration count; CG loops under -iters. `kernels`: the
  // kernel nodes of the captured graph (those of child graphs included).
  struct CachedGraph {
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
  };
  std::map<int, CachedGraph> graphs;
};

namespace ash {

// The handle's executable graph for `key` (a WGS iteration count, or minus a
// CG iteration count): on first use, body(h, iters, capture stream) is
// captured, instantiated and cached with its kernel-node count.
ash_status cached_graph(ash_hologram* h, int key, ash_status (*body)(ash_hologram*, int, cudaStream_t), int iters,
                        cudaGraphExec_t* exec);
// Drop every cached graph (options or shapes they captured have changed).
void clear_graphs(ash_hologram* h);
// Kernel nodes of a graph, those of embedded child graphs included (-1 if
// the graph cannot be inspected).
int graph_kernel_nodes(cudaGraph_t g);
// The FMA-pipe kernels' register-image basis: rebuilt from the monomial
// tables if it was released (synchronises the device).
ash_status ensure_fma_image(ash_hologram* h);
// Record a message for ash_last_error() (any translation unit).
void record_error(const char* msg);
// Map a CUDA error to ASH_ERR_CUDA with a message.
ash_status status_cuda(cudaError_t e, const char* where);
// Host-side fault injection counter (ash_debug_fail_after).
bool consume_injected_failure();
// The single-hologram WGS loop on the handle's state buffers (wgs_phase,
// wgs_w, wgs_T; metrics to wgs_metrics), enqueued on `s`: for callers that
// capture it into a graph of their own (the batched form's standalone
// members).
ash_status wgs_body(ash_hologram* h, int iters, cudaStream_t s);
// The transforms and the coefficient images of a handle, enqueued on `s`
// (for the translation units of the loops built on them).
ash_status forward_enqueue(ash_hologram* h, int source, const float* phase, const float2* field, float2* E,
                           cudaStream_t s);
ash_status adjoint_enqueue(ash_hologram* h, const float2* y, float2* g_out, float* phase_out, const float* phase_in,
                           float* dphase, int epilogue, cudaStream_t s);
cudaError_t coeff_images_enqueue(ash_hologram* h, cudaStream_t s);
// CG workspace: fp64 scalar slots, reduction partials, iterations per call.
constexpr int kCgSlots = 13, kCgRedBlocks = 512, kCgMaxIters = 1024;

inline HoloView view_of(const ash_hologram* h) {
  HoloView v{};
  v.g = h->g;
  v.dz = h->dz;
  v.amp_img = h->amp_img;
  v.anchors = h->anchors;
  v.coeff = h->coeff;
  return v;
}

}  // namespace ash
