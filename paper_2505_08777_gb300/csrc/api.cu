// C ABI of the library (declared in include/ash.h): argument validation,
// workspace ownership, launch orchestration, and the CUDA-graph WGS loop.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ash.h"
#include "aux_kernels.cuh"
#include "basis_host.h"
#include "handle.h"
#include "launch.h"
#include "tc_common.cuh"
#include "tc_launch.h"

using namespace ash;

namespace {

thread_local std::string g_last_error;

ash_alloc_fn g_alloc = nullptr;
ash_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;
std::mutex g_mu;
int g_fail_after = 0;   // 0 = off

ash_status set_error(ash_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

ash_status cuda_fail(cudaError_t e, const char* where) {
  return set_error(ASH_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define ASH_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// Counts calls that would launch work; returns true if this one is injected to fail.
bool injected_failure() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_fail_after <= 0) return false;
  if (--g_fail_after == 0) return true;
  return false;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

namespace ash {
// Lets other translation units report through ash_last_error().
void record_error(const char* msg) { g_last_error = msg; }
ash_status status_invalid(const char* msg) { return set_error(ASH_ERR_INVALID_ARG, "%s", msg); }
ash_status status_cuda(cudaError_t e, const char* where) { return cuda_fail(e, where); }
bool consume_injected_failure() { return injected_failure(); }
}  // namespace ash


namespace {

ash_status ws_alloc(ash_hologram* h, void** out, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (g_alloc) {
    p = g_alloc(g_alloc_ctx, bytes, h->home);
    if (!p) return set_error(ASH_ERR_OOM, "allocator hook returned NULL for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, h->home);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(ASH_ERR_OOM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  h->allocs.push_back(p);
  h->bytes += bytes;
  *out = p;
  return ASH_OK;
}

template <typename T>
ash_status ws(ash_hologram* h, T** out, size_t count) {
  return ws_alloc(h, reinterpret_cast<void**>(out), count * sizeof(T));
}

void free_one(ash_hologram* h, void* p, size_t bytes) {
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i] == p) {
      h->allocs.erase(h->allocs.begin() + (long)i);
      break;
    }
  if (g_free) g_free(g_alloc_ctx, p, h->home);
  else cudaFreeAsync(p, h->home);
  h->bytes -= (bytes + 255) & ~(size_t)255;
}

size_t fma_image_bytes(const ash_hologram* h) { return (size_t)h->g.T * kTilePix * h->g.D * sizeof(float); }

void drop_fma_image(ash_hologram* h) {
  if (!h->dz) return;
  free_one(h, h->dz, fma_image_bytes(h));
  h->dz = nullptr;
}

void release(ash_hologram* h) {
  ash::clear_graphs(h);
  for (void* p : h->allocs) {
    if (g_free) g_free(g_alloc_ctx, p, h->home);
    else cudaFreeAsync(p, h->home);
  }
  h->allocs.clear();
  if (h->capture) cudaStreamDestroy(h->capture);
  h->capture = nullptr;
}

cudaError_t prepare(int D, LaunchInfo* li) {
  switch (range_of(D)) {
    case 0: return prepare_r0(D, li);
    case 1: return prepare_r1(D, li);
    case 2: return prepare_r2(D, li);
    case 3: return prepare_r3(D, li);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_forward(int D, const FwdParams& p, int grid, cudaStream_t s) {
  switch (range_of(D)) {
    case 0: return launch_forward_r0(D, p, grid, s);
    case 1: return launch_forward_r1(D, p, grid, s);
    case 2: return launch_forward_r2(D, p, grid, s);
    case 3: return launch_forward_r3(D, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint(int D, const AdjParams& p, int grid, cudaStream_t s) {
  switch (range_of(D)) {
    case 0: return launch_adjoint_r0(D, p, grid, s);
    case 1: return launch_adjoint_r1(D, p, grid, s);
    case 2: return launch_adjoint_r2(D, p, grid, s);
    case 3: return launch_adjoint_r3(D, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

// Kernel family per transform. Automatic: the tensor-core kernels where an
// operand row fits one 128-byte K-atom (D <= 10) and there are enough spots
// for their chunks of 64 (measured on GB300: the tensor-core forward is
// faster from N = 64, the tensor-core adjoint from N = 256 -- below that a
// partial last spot chunk costs it more than the FMA kernel); the FMA-pipe
// kernels otherwise. Variant 1 / 2 force one family (2 needs D <= 21).
constexpr int kTcFwdMinSpots = 64, kTcAdjMinSpots = 256;
bool use_tc_fwd(const ash_hologram* h) {
  if (!h->tc_ok || h->variant == 1) return false;
  return h->variant == 2 || (h->tc_na == 1 && h->g.N >= kTcFwdMinSpots);
}
bool use_tc_adj(const ash_hologram* h) {
  if (!h->tc_ok || h->variant == 1) return false;
  return h->variant == 2 || (h->tc_na == 1 && h->g.N >= kTcAdjMinSpots);
}
// The coefficient-gradient moments on the tensor cores need one K-atom,
// D <= 12 and a polynomial basis of total degree <= 4 (the tile polynomials);
// from N = 64, as the forward whose structure they share.
bool use_tc_grad(const ash_hologram* h) {
  if (!h->tgrad_ok || h->variant == 1) return false;
  return h->variant == 2 || h->g.N >= kTcFwdMinSpots;
}

// Whether the handle's current kernel choice runs any FMA-pipe kernel (they
// read the register-image basis dz; the tensor-core kernels do not).
bool needs_fma_image(const ash_hologram* h) { return !(use_tc_fwd(h) && use_tc_adj(h) && use_tc_grad(h)); }

// CTA range starts that give every CTA the same estimated time rather than
// the same number of units: prefix(u) is the summed cost of units [0, u)
// (non-decreasing); begin[g] is the first unit at which it reaches g / G of
// the total.
template <typename F>
std::vector<long long> balanced_begins(long long units, int G, F prefix) {
  std::vector<long long> b((size_t)G + 1);
  const double total = prefix(units);
  b[0] = 0;
  b[G] = units;
  for (int g = 1; g < G; ++g) {
    const double target = total * g / G;
    long long lo = b[g - 1], hi = units;
    while (lo < hi) {
      const long long mid = lo + (hi - lo) / 2;
      if (prefix(mid) >= target) hi = mid;
      else lo = mid + 1;
    }
    b[g] = lo;
  }
  return b;
}

// Relative cost of the transforms' cheaper units. The adjoint's last spot
// chunk of a group, with v of its 64 columns valid, costs about
// 0.3 + 0.7 v / 64 of a full chunk (its MMA, barriers and TMEM loads are
// paid whatever v is): weighting it so gave the c3 adjoint (N = 2000,
// v = 16) 2800 us against 2841 with equal ranges (0.2: 2796, 0.45: 2818).
// A chunk of the forward's replicated last spot block has a quarter or a
// half of a full chunk's arithmetic per warp, but the CTAs that run them
// are bound by the MMA pipeline: weighting them 0.4 / 0.55 / 0.7 made the
// c2 forward 380 / 316 / 287 us against 267 with equal ranges, so they
// count as full chunks.
#ifndef ASH_FWD_REP4_COST
#define ASH_FWD_REP4_COST 1.0
#endif
#ifndef ASH_FWD_REP2_COST
#define ASH_FWD_REP2_COST 1.0
#endif
#ifndef ASH_ADJ_TAIL_FIXED
#define ASH_ADJ_TAIL_FIXED 0.3
#endif

TcGradParams tc_grad_params(const ash_hologram* h, const float2* gE, float* dC) {
  TcGradParams p{};
  p.g = h->g;
  p.zs = h->zs;
  p.czs = h->czs;
  p.rot = h->rot;
  p.fimg = h->fimg;
  p.tpoly = h->tpoly;
  p.ord = h->tgrad_ord;
  p.gE = gE;
  p.sched = h->tgrad;
  p.begin = h->tgrad_begin;
  p.spans = h->tgrad_spans;
  p.dC = dC;
  p.part = h->tgrad_part;
  p.err = h->err_word;
  return p;
}

// dC through the tensor-core moment pass: nearfield image of `phase`, then
// the moments (and the sums of split spot blocks).
cudaError_t enqueue_tc_gradc(ash_hologram* h, const float* phase, const float2* gE, float* dC, cudaStream_t s) {
  cudaError_t e = tc_field_img(h->g, h->amp_img, phase, nullptr, h->fimg, s);
  if (e != cudaSuccess) return e;
  return tc_launch_gradc(tc_grad_params(h, gE, dC), h->tgrad_split, s);
}

// Source of a forward: a phase or a complex field in user layout, or the
// tc-layout nearfield the previous tensor-core adjoint wrote (kEpiFimg).
constexpr int kSrcImg = 2;

cudaError_t enqueue_tc_coeff(ash_hologram* h, cudaStream_t s) {
  if (!h->tc_ok) return cudaSuccess;
  return tc_build_coeff(h->g, h->tc_layout, h->coeff, h->anchors, h->czs, h->rot, s);
}

TcFwdParams tc_fwd_params(const ash_hologram* h, float2* E) {
  TcFwdParams p{};
  p.g = h->g;
  p.zs = h->zs;
  p.czs = h->czs;
  p.rot = h->rot;
  p.fimg = h->fimg;
  p.sched = h->tfwd;
  p.rep = tc_fwd_rep(h->g.N);
  p.begin = h->tfwd_begin;
  p.E = E;
  p.part = h->tc_part;
  p.spans = h->tfwd_spans;
  p.err = h->err_word;
  p.claim = h->tfwd_nfull >= 0 ? h->tfwd_claim : nullptr;
  p.n_full = h->tfwd_nfull;
  return p;
}

TcAdjParams tc_adj_params(const ash_hologram* h, const float2* y, const AdjOut& out) {
  TcAdjParams p{};
  p.g = h->g;
  p.zs = h->zs;
  p.czs = h->czs;
  p.rot = h->rot;
  p.y = y;
  p.amp_img = h->amp_img;
  p.out = out;
  p.fimg = h->fimg;
  p.begin = h->tadj_begin;
  p.G = h->tadj.G;
  p.split = h->tc_split;
  p.split_groups = h->tadj_groups;
  p.err = h->err_word;
  return p;
}

cudaError_t launch_gradc(int D, const GradCParams& p, dim3 grid, cudaStream_t s) {
  switch (range_of(D)) {
    case 0: return launch_gradc_r0(D, p, grid, s);
    case 1: return launch_gradc_r1(D, p, grid, s);
    case 2: return launch_gradc_r2(D, p, grid, s);
    case 3: return launch_gradc_r3(D, p, grid, s);
  }
  return cudaErrorInvalidValue;
}

// forward transform into E (device complex [N]).
ash_status enqueue_forward(ash_hologram* h, int source, const float* phase, const float2* field, float2* E,
                           cudaStream_t s) {
  if (use_tc_fwd(h)) {
    cudaError_t e = cudaSuccess;
    if (source != kSrcImg) {
      e = tc_field_img(h->g, h->amp_img, source == kSrcPhase ? phase : nullptr, field, h->fimg, s);
      if (e != cudaSuccess) return cuda_fail(e, "nearfield image launch");
    }
    const TcFwdParams tp = tc_fwd_params(h, E);
    e = tc_launch_forward(h->tc_na, tp, h->tfwd.G, s);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core forward launch");
    if (h->tfwd_split) {
      e = tc_launch_forward_reduce(tp, s);
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core forward reduce launch");
    }
    return ASH_OK;
  }
  if (!h->dz) return set_error(ASH_ERR_DEVICE, "FMA-pipe forward without its basis image");
  FwdParams p{};
  p.v = view_of(h);
  p.phase = phase;
  p.field = field;
  p.source = source;
  p.sched = h->sched;
  p.partial = h->partial;
  cudaError_t e = launch_forward(h->g.D, p, h->sched.G, s);
  if (e != cudaSuccess) return cuda_fail(e, "forward kernel launch");
  const int cols = 2 * h->g.N;
  k_col_reduce<<<(cols + 31) / 32, dim3(32, 32), 0, s>>>(h->partial, h->fwd_rows, cols, reinterpret_cast<float*>(E));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "forward reduce launch");
  return ASH_OK;
}

ash_status enqueue_adjoint(ash_hologram* h, const float2* y, float2* g_out, float* phase_out, const float* phase_in,
                           float* dphase, int epilogue, cudaStream_t s) {
  AdjParams p{};
  p.v = view_of(h);
  p.y = y;
  p.out.g_out = g_out;
  p.out.phase_out = phase_out;
  p.out.phase_in = phase_in;
  p.out.dphase = dphase;
  p.out.epilogue = epilogue;
  if (use_tc_adj(h)) {
    const TcAdjParams tp = tc_adj_params(h, y, p.out);
    cudaError_t e = tc_launch_adjoint(h->tc_na, tp, h->tadj.G, s);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core adjoint launch");
    if (h->tadj_split) {
      e = tc_launch_adjoint_fixup(tp, h->tadj_nsplit, s);
      if (e != cudaSuccess) return cuda_fail(e, "tensor-core adjoint fix-up launch");
    }
    return ASH_OK;
  }
  if (!h->dz) return set_error(ASH_ERR_DEVICE, "FMA-pipe adjoint without its basis image");
  p.sched = h->sched;
  p.split = h->split;
  cudaError_t e = launch_adjoint(h->g.D, p, h->sched.G, s);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel launch");
  if (h->split_tiles) {
    k_adjoint_fixup<<<h->g.T, h->g.NT, 0, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint fix-up launch");
  }
  return ASH_OK;
}

// iters x (forward, spot update, adjoint), then a final forward and the
// metrics. When both transforms run on the tensor cores the adjoint also
// writes the next forward's nearfield (kEpiFimg), so only the first forward
// converts a phase.
bool wgs_fused_field(const ash_hologram* h) { return use_tc_fwd(h) && use_tc_adj(h); }

ash_status enqueue_wgs_body(ash_hologram* h, int iters, cudaStream_t s) {
  const bool tc = wgs_fused_field(h);
  const int adj_epi = tc ? (kEpiPhase | kEpiFimg) : kEpiPhase;
  ash_status st = enqueue_forward(h, kSrcPhase, h->wgs_phase, nullptr, h->wgs_E, s);
  if (st != ASH_OK) return st;
  for (int it = 0; it < iters; ++it) {
    k_wgs_update<<<1, 1024, 0, s>>>(h->wgs_E, h->wgs_w, h->wgs_T, h->y, h->g.N, h->wgs_feedback,
                                    h->wgs_fix ? h->wgs_u : nullptr, h->wgs_fix ? nullptr : h->wgs_u);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "wgs update launch");
    st = enqueue_adjoint(h, h->y, nullptr, h->wgs_phase, nullptr, nullptr, adj_epi, s);
    if (st != ASH_OK) return st;
    st = enqueue_forward(h, tc ? kSrcImg : kSrcPhase, h->wgs_phase, nullptr, h->wgs_E, s);
    if (st != ASH_OK) return st;
  }
  k_metrics<<<1, 1024, 0, s>>>(h->wgs_E, h->wgs_T, h->g.N, h->sum_a2, (double)h->g.nx * h->g.ny, h->wgs_metrics);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "metrics launch");
  return ASH_OK;
}

bool bad_ptr(const void* p) { return p == nullptr; }

}  // namespace

namespace ash {

ash_status ensure_fma_image(ash_hologram* h) {
  if (h->dz) return ASH_OK;
  // work in flight may use the handle; the image is rebuilt with the device idle
  ASH_CUDA(cudaDeviceSynchronize());
  ash_status st = ws(h, &h->dz, (size_t)h->g.T * kTilePix * h->g.D);
  if (st != ASH_OK) return st;
  BasisParams bp{};
  bp.g = h->g;
  bp.terms = h->terms;
  bp.term_off = h->term_off;
  bp.max_order = h->basis_max_order;
  bp.dz = h->dz;
  bp.anchors = nullptr;   // the anchors are kept; only the image is rebuilt
  k_basis<<<h->g.T, h->g.NT, 0, h->home>>>(bp);
  ASH_CUDA(cudaGetLastError());
  ASH_CUDA(cudaStreamSynchronize(h->home));
  return ASH_OK;
}

int graph_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
  int k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess) return -1;
    if (t == cudaGraphNodeTypeKernel) {
      ++k;
    } else if (t == cudaGraphNodeTypeGraph) {
      cudaGraph_t child = nullptr;
      if (cudaGraphChildGraphNodeGetGraph(nd, &child) != cudaSuccess) return -1;
      const int m = graph_kernel_nodes(child);
      if (m < 0) return -1;
      k += m;
    }
  }
  return k;
}

ash_status cached_graph(ash_hologram* h, int key, ash_status (*body)(ash_hologram*, int, cudaStream_t), int iters,
                        cudaGraphExec_t* exec) {
  auto it = h->graphs.find(key);
  if (it != h->graphs.end()) {
    *exec = it->second.exec;
    return ASH_OK;
  }
  cudaGraph_t graph = nullptr;
  ASH_CUDA(cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal));
  ash_status st = body(h, iters, h->capture);
  cudaError_t ce = cudaStreamEndCapture(h->capture, &graph);
  if (st != ASH_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
  ash_hologram::CachedGraph c;
  c.kernels = graph_kernel_nodes(graph);
  ce = cudaGraphInstantiate(&c.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
  h->graphs[key] = c;
  *exec = c.exec;
  return ASH_OK;
}

void clear_graphs(ash_hologram* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
}

ash_status wgs_body(ash_hologram* h, int iters, cudaStream_t s) { return enqueue_wgs_body(h, iters, s); }
ash_status forward_enqueue(ash_hologram* h, int source, const float* phase, const float2* field, float2* E,
                           cudaStream_t s) {
  return enqueue_forward(h, source, phase, field, E, s);
}
ash_status adjoint_enqueue(ash_hologram* h, const float2* y, float2* g_out, float* phase_out, const float* phase_in,
                           float* dphase, int epilogue, cudaStream_t s) {
  return enqueue_adjoint(h, y, g_out, phase_out, phase_in, dphase, epilogue, s);
}
cudaError_t coeff_images_enqueue(ash_hologram* h, cudaStream_t s) { return enqueue_tc_coeff(h, s); }
}  // namespace ash

// A bounded wait that is never released: one thread waits on a fresh
// mbarrier that nothing arrives on, for at most `polls` polls, and then
// reports the timeout in the error word exactly as the transforms do.
static __global__ void k_debug_wait(uint32_t polls, unsigned* __restrict__ err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!mbar_wait(&bar, 0u, polls)) atomicOr(err, kErrTimeout);
    mbar_inval(&bar);
  }
}

// Two pixels per thread, as in the transforms' pair loops.
static __global__ void k_debug_sincos(const float* __restrict__ x, int n, float* __restrict__ s, float* __restrict__ c,
                               int path) {
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  const float2 v = make_float2(x[i], i + 1 < n ? x[i + 1] : 0.0f);
  float2 sn, cs;
  if (path == 1) {
    sincos2_poly(v, sn, cs);
  } else {
    sincos2(v, sn, cs);
  }
  s[i] = sn.x;
  c[i] = cs.x;
  if (i + 1 < n) {
    s[i + 1] = sn.y;
    c[i + 1] = cs.y;
  }
}

extern "C" {

int ash_abi_version(void) { return ASH_ABI_VERSION; }

const char* ash_status_string(ash_status s) {
  switch (s) {
    case ASH_OK: return "ASH_OK";
    case ASH_ERR_INVALID_ARG: return "ASH_ERR_INVALID_ARG";
    case ASH_ERR_CUDA: return "ASH_ERR_CUDA";
    case ASH_ERR_OOM: return "ASH_ERR_OOM";
    case ASH_ERR_TIMEOUT: return "ASH_ERR_TIMEOUT";
    case ASH_ERR_UNSUPPORTED: return "ASH_ERR_UNSUPPORTED";
    case ASH_ERR_INJECTED: return "ASH_ERR_INJECTED";
    case ASH_ERR_DEVICE: return "ASH_ERR_DEVICE";
  }
  return "ASH_ERR_UNKNOWN";
}

const char* ash_last_error(void) { return g_last_error.c_str(); }

ash_status ash_set_allocator(ash_alloc_fn alloc, ash_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return set_error(ASH_ERR_INVALID_ARG, "allocator hook needs both alloc and free (or neither)");
  std::lock_guard<std::mutex> lk(g_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return ASH_OK;
}

ash_status ash_debug_sincos(const float* x, int n, float* s, float* c, int path, void* stream) {
  if (!x || !s || !c || n < 0 || path < 0 || path > 1) return set_error(ASH_ERR_INVALID_ARG, "invalid argument");
  if (n == 0) return ASH_OK;
  k_debug_sincos<<<(n + 255) / 256, 256, 0, as_stream(stream)>>>(x, n, s, c, path);
  ASH_CUDA(cudaGetLastError());
  return ASH_OK;
}

ash_status ash_debug_fail_after(int n_calls) {
  if (n_calls < 0) return set_error(ASH_ERR_INVALID_ARG, "n_calls must be >= 0");
  std::lock_guard<std::mutex> lk(g_mu);
  g_fail_after = n_calls;
  return ASH_OK;
}

}  // extern "C"

namespace {

// The basis of a hologram built from Zernike modes: monomial tables of the
// D output modes (each a fixed combination of Noll-indexed Zernikes), and
// the Noll index of every output mode that is a single Zernike (0 otherwise).
struct BasisSpec {
  std::vector<MonoTerm> terms;
  std::vector<int> off{0};
  std::vector<int> noll_eff;
  int max_order = 0;
};

// Output mode k = sum_d mix[k][d] Z_{noll[d]} (mix = NULL: the identity);
// equal monomials are merged in fp64.
ash_status build_spec(int D_in, const int* noll, int D, const double* mix, BasisSpec* sp) {
  std::vector<std::vector<MonoTerm>> in(D_in);
  std::vector<int> order(D_in);
  for (int d = 0; d < D_in; ++d) {
    int n, m;
    if (noll[d] < 1 || noll[d] > 231 || !noll_to_nm(noll[d], &n, &m))
      return set_error(ASH_ERR_INVALID_ARG, "Noll index %d outside [1, 231]", noll[d]);
    if (!zernike_monomials(n, m, &in[d])) return set_error(ASH_ERR_INVALID_ARG, "bad Zernike (%d, %d)", n, m);
    order[d] = n;
  }
  sp->noll_eff.assign(D, 0);
  for (int k = 0; k < D; ++k) {
    std::map<std::pair<int, int>, double> acc;
    int nz = 0, last = -1;
    for (int d = 0; d < D_in; ++d) {
      const double wgt = mix ? mix[(size_t)k * D_in + d] : (d == k ? 1.0 : 0.0);
      if (wgt == 0.0) continue;
      ++nz;
      last = d;
      sp->max_order = order[d] > sp->max_order ? order[d] : sp->max_order;
      for (const MonoTerm& t : in[d]) acc[{t.px, t.py}] += wgt * t.coef;
    }
    if (nz == 1 && (mix ? mix[(size_t)k * D_in + last] : 1.0) == 1.0) sp->noll_eff[k] = noll[last];
    for (const auto& kv : acc)
      if (kv.second != 0.0) sp->terms.push_back(MonoTerm{kv.second, kv.first.first, kv.first.second});
    sp->off.push_back((int)sp->terms.size());
  }
  return ASH_OK;
}

ash_status create_impl(ash_hologram** out, int nx, int ny, int row0, int ny_full, const float* amp, int D,
                       const BasisSpec* spec, const float* basis, int N, const float* coeff, void* stream) {
  const int* noll = spec ? spec->noll_eff.data() : nullptr;
  const int max_order = spec ? spec->max_order : 0;
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure (ash_debug_fail_after)");

  ash_hologram* h = new ash_hologram();
  cudaStream_t s = as_stream(stream);
  h->home = s;
  cudaGetDevice(&h->device);
  Geometry& g = h->g;
  g.nx = nx;
  g.ny = ny;
  g.tiles_x = (nx + kTileX - 1) / kTileX;
  g.tiles_y = (ny + kTileY - 1) / kTileY;
  g.T = g.tiles_x * g.tiles_y;
  g.D = D;
  g.N = N;
  g.P = pixels_per_thread(D);
  g.NT = kTilePix / g.P;
  g.row0 = row0;
  g.ny_full = ny_full;

  auto fail = [&](ash_status st) {
    release(h);
    delete h;
    return st;
  };
  cudaError_t ce = prepare(D, &h->li);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "kernel preparation"));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  {
    // One range of (tile, spot) units per resident CTA; at least min(256, N)
    // units per CTA so that small problems keep whole tiles together.
    int per_sm = h->li.fwd_ctas_per_sm < h->li.adj_ctas_per_sm ? h->li.fwd_ctas_per_sm : h->li.adj_ctas_per_sm;
    if (per_sm < 1) per_sm = 1;
    const long long W = (long long)g.T * N;
    const long long umin = N < 256 ? N : 256;
    long long G = (long long)sms * per_sm;
    if (G > W / umin) G = W / umin;
    if (G < 1) G = 1;
    h->sched.W = W;
    h->sched.G = (int)G;
    for (int b = 1; b < h->sched.G; ++b)
      if (h->sched.begin(b) % N != 0) h->split_tiles = true;
  }
  h->fwd_rows = g.T * (g.NT / 32);
  std::vector<int4> tadj_groups;
  std::vector<int2> tfwd_spans, tgrad_spans;
  std::vector<long long> tfwd_begin, tadj_begin, tgrad_begin;
  if (D <= kTcMaxModes) {
    // tensor-core path: one range of units per resident CTA, at least two
    // MMA chunks per CTA
    h->tc_layout = tc_layout(D, noll, g);
    h->tc_na = h->tc_layout.NA;
    // the spot-side kernels between tensor-core launches keep the SMs'
    // shared-memory carveout (see tc_small_kernels_max_shared)
    for (const void* k : {(const void*)k_wgs_update, (const void*)k_metrics, (const void*)k_spot_loss,
                          (const void*)k_col_reduce, (const void*)k_fill_c})
      cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    ce = tc_prepare(h->tc_na, &h->li.tc_adj_ctas_per_sm, &h->li.tc_fwd_ctas_per_sm);
    if (ce != cudaSuccess) return fail(cuda_fail(ce, "tensor-core kernel preparation"));
    h->tc_ok = true;
    const int nch = (N + kTcChunk - 1) / kTcChunk;
    const long long Wa = (long long)g.T * kTcGroupsPerTile * nch;
    long long Ga = (long long)sms * h->li.tc_adj_ctas_per_sm;
    if (Ga > Wa / 2) Ga = Wa / 2;
    if (Ga < 1) Ga = 1;
    h->tadj.W = Wa;
    h->tadj.G = (int)Ga;
    {
      const int v = N - kTcChunk * (nch - 1);
      const double tail = nch > 1 ? ASH_ADJ_TAIL_FIXED + (1.0 - ASH_ADJ_TAIL_FIXED) * v / kTcChunk : 1.0;
      tadj_begin = balanced_begins(Wa, h->tadj.G, [&](long long u) {
        return (double)(u / nch) * (nch - 1 + tail) + (double)(u % nch);
      });
    }
    for (int b = 1; b < h->tadj.G; ++b) {
      const long long u = tadj_begin[b];
      if (u % nch == 0) continue;
      const int grp = (int)(u / nch);
      if (tadj_groups.empty() || tadj_groups.back().x != grp) {
        const long long ulo = (long long)grp * nch;
        tadj_groups.push_back(make_int4(grp, tc_owner(tadj_begin.data(), h->tadj.G, ulo),
                                        tc_owner(tadj_begin.data(), h->tadj.G, ulo + nch - 1), 0));
      }
    }
    h->tadj_split = !tadj_groups.empty();
    h->tadj_nsplit = (int)tadj_groups.size();
    TcFwdSched& f = h->tfwd;
    f.nb = (N + kTcRows - 1) / kTcRows;
    f.nq = g.T * kTcChunksPerTile;
    long long Gf = (long long)sms * h->li.tc_fwd_ctas_per_sm;
    if (Gf > f.units() / 2) Gf = f.units() / 2;
    if (Gf < 1) Gf = 1;
    f.G = (int)Gf;
    {
      const int rep = tc_fwd_rep(N);
      const double cheap = rep == 4 ? ASH_FWD_REP4_COST : rep == 2 ? ASH_FWD_REP2_COST : 1.0;
      const long long u_rep = (long long)(f.nb - 1) * f.nq;
      const int per_sm = h->li.tc_fwd_ctas_per_sm;
      h->tfwd_nfull = -1;
      if (rep > 1 && f.nb >= 2 && per_sm >= 2 && f.G == sms * per_sm && sms <= kTcClaimSms &&
          f.units() >= 32LL * f.G) {
        // a replicated last block: one of its ranges per SM, claimed by each
        // SM's last CTA (tc_claim_range), the full blocks' in the others.
        // Only for ranges of 32 chunks or more: claiming costs about 2 us
        // per launch, a tenth of a small forward.
        const int n_full = f.G - sms;
        tfwd_begin = balanced_begins(u_rep, n_full, [](long long u) { return (double)u; });
        const std::vector<long long> tail = balanced_begins(f.nq, sms, [](long long u) { return (double)u; });
        for (int k = 1; k <= sms; ++k) tfwd_begin.push_back(u_rep + tail[k]);
        h->tfwd_nfull = n_full;
      } else {
        tfwd_begin = balanced_begins(f.units(), f.G, [&](long long u) {
          return (double)(u < u_rep ? u : u_rep) + cheap * (double)(u > u_rep ? u - u_rep : 0);
        });
      }
    }
    for (int b = 1; b < f.G; ++b)
      if (tfwd_begin[b] % f.nq != 0) h->tfwd_split = true;
    for (int b = 0; b < f.nb; ++b) {
      const long long ulo = (long long)b * f.nq;
      tfwd_spans.push_back(make_int2(tc_owner(tfwd_begin.data(), f.G, ulo), tc_owner(tfwd_begin.data(), f.G, ulo + f.nq - 1)));
    }
    int ord = 1;
    if (spec)
      for (const MonoTerm& m : spec->terms) ord = m.px + m.py > ord ? m.px + m.py : ord;
    if (spec && h->tc_na == 1 && D <= kTcGradMaxModes && ord <= kTcGradMaxOrd) {
      h->tgrad_ord = ord;
      ce = tc_grad_prepare(ord, D, &h->li.tc_grad_ctas_per_sm);
      if (ce != cudaSuccess) return fail(cuda_fail(ce, "tensor-core moment pass preparation"));
      h->tgrad_ok = true;
      TcFwdSched& m = h->tgrad;
      m.nb = f.nb;
      m.nq = f.nq;
      long long Gm = (long long)sms * h->li.tc_grad_ctas_per_sm;
      if (Gm > m.units() / 2) Gm = m.units() / 2;
      if (Gm < 1) Gm = 1;
      m.G = (int)Gm;
      for (int b = 0; b <= m.G; ++b) tgrad_begin.push_back(m.begin(b));
      for (int b = 1; b < m.G; ++b)
        if (tgrad_begin[b] % m.nq != 0) h->tgrad_split = true;
      for (int b = 0; b < m.nb; ++b) {
        const long long ulo = (long long)b * m.nq;
        tgrad_spans.push_back(
            make_int2(tc_owner(tgrad_begin.data(), m.G, ulo), tc_owner(tgrad_begin.data(), m.G, ulo + m.nq - 1)));
      }
    }
  }
  h->gradc_gy = (N + kGradThreads * kGradSpots - 1) / (kGradThreads * kGradSpots);
  {
    const int slots = sms * (h->li.gradc_ctas_per_sm > 0 ? h->li.gradc_ctas_per_sm : 1);
    int gx = slots / h->gradc_gy;
    if (gx < 1) gx = 1;
    if (gx > g.T) gx = g.T;
    h->gradc_gx = gx;
  }
  const size_t M = (size_t)nx * ny;
  const size_t pix = (size_t)g.T * kTilePix;
  ash_status st;
  if ((st = ws(h, &h->dz, pix * D)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->amp_img, pix)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->anchors, (size_t)g.T * D)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->coeff, (size_t)N * D)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->coeff_bak, (size_t)N * D)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->partial, (size_t)h->fwd_rows * 2 * N)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->split, (size_t)h->sched.G * 2 * kTilePix)) != ASH_OK) return fail(st);
  if (h->tc_ok) {
    if ((st = ws(h, &h->zs, tc_zs_floats(g, h->tc_na))) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->czs, tc_czs_floats(N, h->tc_na))) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->fimg, tc_fimg_float4s(g))) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->rot, (size_t)N * g.T)) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tc_split, (size_t)h->tadj.G * 2 * kTcRows)) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tc_part, (size_t)h->tfwd.G * 2 * kTcRows)) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tfwd_begin, tfwd_begin.size())) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tfwd_spans, tfwd_spans.size())) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tfwd_claim, (size_t)kTcClaimInts)) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tadj_begin, tadj_begin.size())) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tadj_groups, tadj_groups.size() + 1)) != ASH_OK) return fail(st);
  }
  if (h->tgrad_ok) {
    if ((st = ws(h, &h->tpoly, tc_tpoly_floats(g, h->tgrad_ord))) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tgrad_part, (size_t)h->tgrad.G * 2 * kTcRows * tc_grad_dp(D))) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tgrad_begin, tgrad_begin.size())) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->tgrad_spans, tgrad_spans.size())) != ASH_OK) return fail(st);
  }
  if ((st = ws(h, &h->gradc_partial, (size_t)h->gradc_gx * N * D)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->E, (size_t)N)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->y, (size_t)N)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->wgs_phase, M)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->wgs_w, (size_t)N)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->wgs_T, (size_t)N)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->wgs_E, (size_t)N)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->wgs_u, (size_t)N)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->wgs_metrics, 4)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->cg_phase, M)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->cg_t, (size_t)N)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->cg_g, 2 * M)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->cg_d, M)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->cg_trial, M)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->cg_scal, kCgSlots)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->cg_part, kCgRedBlocks)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->cg_loss, kCgMaxIters + 1)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->sum_a2, 1)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->sum_a2_arg, 1)) != ASH_OK) return fail(st);
  if ((st = ws(h, &h->err_word, 1)) != ASH_OK) return fail(st);
  if (spec) {
    if ((st = ws(h, &h->terms, spec->terms.size() + 1)) != ASH_OK) return fail(st);
    if ((st = ws(h, &h->term_off, spec->off.size())) != ASH_OK) return fail(st);
  }
  ce = cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return fail(cuda_fail(ce, "capture stream"));

#define CREATE_CUDA(call)                                     \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return fail(cuda_fail(e_, #call)); \
  } while (0)
  if (spec) {
    if (!spec->terms.empty())
      CREATE_CUDA(cudaMemcpyAsync(h->terms, spec->terms.data(), spec->terms.size() * sizeof(MonoTerm),
                                  cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemcpyAsync(h->term_off, spec->off.data(), spec->off.size() * sizeof(int), cudaMemcpyHostToDevice,
                                s));
  }
  CREATE_CUDA(cudaMemsetAsync(h->err_word, 0, sizeof(unsigned), s));
  // stored spot phases of the phase-fixing variant start at 0
  k_fill_c<<<(N + 255) / 256, 256, 0, s>>>(h->wgs_u, N, make_float2(1.0f, 0.0f));
  CREATE_CUDA(cudaGetLastError());
  CREATE_CUDA(cudaMemcpyAsync(h->coeff, coeff, (size_t)N * D * sizeof(float), cudaMemcpyDeviceToDevice, s));
  BasisParams bp{};
  bp.g = g;
  bp.terms = h->terms;
  bp.term_off = h->term_off;
  bp.max_order = max_order;
  bp.user_basis = basis;
  bp.dz = h->dz;
  bp.anchors = h->anchors;
  k_basis<<<g.T, g.NT, 0, s>>>(bp);
  CREATE_CUDA(cudaGetLastError());
  h->basis_max_order = max_order;
  h->user_basis = basis != nullptr;
  if (h->tc_ok) {
    CREATE_CUDA(cudaMemcpyAsync(h->tfwd_begin, tfwd_begin.data(), tfwd_begin.size() * sizeof(long long),
                                cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemcpyAsync(h->tfwd_spans, tfwd_spans.data(), tfwd_spans.size() * sizeof(int2),
                                cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemsetAsync(h->tfwd_claim, 0, (size_t)kTcClaimInts * sizeof(int), s));
    CREATE_CUDA(cudaMemcpyAsync(h->tadj_begin, tadj_begin.data(), tadj_begin.size() * sizeof(long long),
                                cudaMemcpyHostToDevice, s));
    if (!tadj_groups.empty())
      CREATE_CUDA(cudaMemcpyAsync(h->tadj_groups, tadj_groups.data(), tadj_groups.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, s));
    CREATE_CUDA(tc_build_zs(g, h->tc_layout, h->dz, h->zs, s));
    if (h->tgrad_ok) {
      CREATE_CUDA(cudaMemcpyAsync(h->tgrad_begin, tgrad_begin.data(), tgrad_begin.size() * sizeof(long long),
                                  cudaMemcpyHostToDevice, s));
      CREATE_CUDA(cudaMemcpyAsync(h->tgrad_spans, tgrad_spans.data(), tgrad_spans.size() * sizeof(int2),
                                  cudaMemcpyHostToDevice, s));
      CREATE_CUDA(tc_build_tile_poly(g, h->terms, h->term_off, h->tgrad_ord, h->tpoly, s));
    }
    // pixels outside the grid stay 0 in every nearfield image
    CREATE_CUDA(cudaMemsetAsync(h->fimg, 0, tc_fimg_float4s(g) * sizeof(float4), s));
  }
  CREATE_CUDA(enqueue_tc_coeff(h, s));
  k_amp_image<<<g.T, g.NT, 0, s>>>(g, amp, h->amp_img);
  CREATE_CUDA(cudaGetLastError());
  k_sum_sq<<<1, 1024, 0, s>>>(amp, M, h->sum_a2);
  CREATE_CUDA(cudaGetLastError());
  // stream-ordered allocations and set-up must be complete before the handle
  // is used from another stream (the graph capture stream, or the caller's)
  CREATE_CUDA(cudaStreamSynchronize(s));
#undef CREATE_CUDA
  // the register-image basis serves only the FMA-pipe kernels: when every
  // transform of this handle runs on the tensor cores, it is released (and
  // rebuilt from the monomial tables if a later kernel choice needs it; a
  // caller's basis is not kept, so its image stays)
  if (!h->user_basis && !needs_fma_image(h)) drop_fma_image(h);
  *out = h;
  return ASH_OK;
}

}  // namespace

extern "C" {

ash_status ash_hologram_create(ash_hologram** out, int nx, int ny, const float* amp, int D, const int* noll,
                               const float* basis, int N, const float* coeff, void* stream) {
  if (!out) return set_error(ASH_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nx > 16384 || ny > 16384)
    return set_error(ASH_ERR_INVALID_ARG, "grid %dx%d outside [1, 16384]", nx, ny);
  if (D < 1 || D > ASH_MAX_MODES) return set_error(ASH_ERR_INVALID_ARG, "D=%d outside [1, %d]", D, ASH_MAX_MODES);
  if (N < 1 || N > (1 << 20)) return set_error(ASH_ERR_INVALID_ARG, "N=%d outside [1, 2^20]", N);
  if (bad_ptr(amp) || bad_ptr(coeff)) return set_error(ASH_ERR_INVALID_ARG, "amp and coeff must be device pointers");
  if ((noll == nullptr) == (basis == nullptr))
    return set_error(ASH_ERR_INVALID_ARG, "exactly one of noll / basis must be given");
  if (!noll) return create_impl(out, nx, ny, 0, ny, amp, D, nullptr, basis, N, coeff, stream);
  BasisSpec spec;
  ash_status st = build_spec(D, noll, D, nullptr, &spec);
  if (st != ASH_OK) return st;
  return create_impl(out, nx, ny, 0, ny, amp, D, &spec, nullptr, N, coeff, stream);
}

ash_status ash_hologram_create_mixed(ash_hologram** out, int nx, int ny, const float* amp, int D_in, const int* noll,
                                     int D, const double* mix, int N, const float* coeff, void* stream) {
  if (!out) return set_error(ASH_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nx > 16384 || ny > 16384)
    return set_error(ASH_ERR_INVALID_ARG, "grid %dx%d outside [1, 16384]", nx, ny);
  if (D_in < 1 || D_in > 64) return set_error(ASH_ERR_INVALID_ARG, "D_in=%d outside [1, 64]", D_in);
  if (D < 1 || D > ASH_MAX_MODES) return set_error(ASH_ERR_INVALID_ARG, "D=%d outside [1, %d]", D, ASH_MAX_MODES);
  if (N < 1 || N > (1 << 20)) return set_error(ASH_ERR_INVALID_ARG, "N=%d outside [1, 2^20]", N);
  if (bad_ptr(amp) || bad_ptr(coeff) || !noll || !mix)
    return set_error(ASH_ERR_INVALID_ARG, "amp, coeff (device), noll and mix (host) must be given");
  BasisSpec spec;
  ash_status st = build_spec(D_in, noll, D, mix, &spec);
  if (st != ASH_OK) return st;
  return create_impl(out, nx, ny, 0, ny, amp, D, &spec, nullptr, N, coeff, stream);
}

ash_status ash_hologram_create_band(ash_hologram** out, int nx, int ny_full, int row0, int row1, const float* amp,
                                    int D, const int* noll, const float* basis, int N, const float* coeff,
                                    void* stream) {
  if (!out) return set_error(ASH_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny_full < 1 || nx > 16384 || ny_full > 16384)
    return set_error(ASH_ERR_INVALID_ARG, "grid %dx%d outside [1, 16384]", nx, ny_full);
  if (row0 < 0 || row1 <= row0 || row1 > ny_full)
    return set_error(ASH_ERR_INVALID_ARG, "band rows [%d, %d) outside [0, %d) or empty", row0, row1, ny_full);
  if (row0 % kTileY != 0 || (row1 % kTileY != 0 && row1 != ny_full))
    return set_error(ASH_ERR_INVALID_ARG, "band rows [%d, %d) must start and end on whole %d-row tile rows", row0,
                     row1, kTileY);
  if (D < 1 || D > ASH_MAX_MODES) return set_error(ASH_ERR_INVALID_ARG, "D=%d outside [1, %d]", D, ASH_MAX_MODES);
  if (N < 1 || N > (1 << 20)) return set_error(ASH_ERR_INVALID_ARG, "N=%d outside [1, 2^20]", N);
  if (bad_ptr(amp) || bad_ptr(coeff)) return set_error(ASH_ERR_INVALID_ARG, "amp and coeff must be device pointers");
  if ((noll == nullptr) == (basis == nullptr))
    return set_error(ASH_ERR_INVALID_ARG, "exactly one of noll / basis must be given");
  const int ny = row1 - row0;
  if (!noll) return create_impl(out, nx, ny, row0, ny_full, amp, D, nullptr, basis, N, coeff, stream);
  BasisSpec spec;
  ash_status st = build_spec(D, noll, D, nullptr, &spec);
  if (st != ASH_OK) return st;
  return create_impl(out, nx, ny, row0, ny_full, amp, D, &spec, nullptr, N, coeff, stream);
}

ash_status ash_hologram_band(const ash_hologram* h, int* row0, int* ny_full, double* sum_a2) {
  if (!h) return set_error(ASH_ERR_INVALID_ARG, "handle is NULL");
  if (row0) *row0 = h->g.row0;
  if (ny_full) *ny_full = h->g.ny_full;
  if (sum_a2) {
    ASH_CUDA(cudaMemcpy(sum_a2, h->sum_a2, sizeof(double), cudaMemcpyDeviceToHost));
  }
  return ASH_OK;
}

ash_status ash_spot_update(ash_hologram* h, const float* E, float* w, const float* target, float* y, void* stream) {
  if (!h || !E || !w || !target || !y) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(E) & 7) || (reinterpret_cast<uintptr_t>(y) & 7))
    return set_error(ASH_ERR_INVALID_ARG, "complex buffers must be 8-byte aligned");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  k_wgs_update<<<1, 1024, 0, as_stream(stream)>>>(reinterpret_cast<const float2*>(E), w, target,
                                                  reinterpret_cast<float2*>(y), h->g.N, h->wgs_feedback,
                                                  h->wgs_fix ? h->wgs_u : nullptr, h->wgs_fix ? nullptr : h->wgs_u);
  ASH_CUDA(cudaGetLastError());
  return ASH_OK;
}

ash_status ash_spot_metrics(ash_hologram* h, const float* E, const float* target, double sum_a2, float* metrics_out,
                            void* stream) {
  if (!h || !E || !target || !metrics_out) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (reinterpret_cast<uintptr_t>(E) & 7) return set_error(ASH_ERR_INVALID_ARG, "E must be 8-byte aligned");
  if (!(sum_a2 >= 0.0)) return set_error(ASH_ERR_INVALID_ARG, "sum_a2 must be >= 0 (0: the handle's own)");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = as_stream(stream);
  const double* sa = h->sum_a2;
  if (sum_a2 > 0.0) {
    // the caller's total sum A^2 (e.g. over every band of a sharded grid)
    ASH_CUDA(cudaMemcpyAsync(h->sum_a2_arg, &sum_a2, sizeof(double), cudaMemcpyHostToDevice, s));
    sa = h->sum_a2_arg;
  }
  k_metrics<<<1, 1024, 0, s>>>(reinterpret_cast<const float2*>(E), target, h->g.N, sa,
                               (double)h->g.nx * h->g.ny_full, metrics_out);
  ASH_CUDA(cudaGetLastError());
  return ASH_OK;
}

void ash_hologram_destroy(ash_hologram* h) {
  if (!h) return;
  // work enqueued on any stream may still read the workspace
  cudaDeviceSynchronize();
  release(h);
  delete h;
}

ash_status ash_hologram_info(const ash_hologram* h, int* nx, int* ny, int* N, int* D, size_t* workspace_bytes) {
  if (!h) return set_error(ASH_ERR_INVALID_ARG, "handle is NULL");
  if (nx) *nx = h->g.nx;
  if (ny) *ny = h->g.ny;
  if (N) *N = h->g.N;
  if (D) *D = h->g.D;
  if (workspace_bytes) *workspace_bytes = h->bytes;
  return ASH_OK;
}

ash_status ash_set_coefficients(ash_hologram* h, const float* coeff, void* stream) {
  if (!h || !coeff) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  ASH_CUDA(cudaMemcpyAsync(h->coeff, coeff, (size_t)h->g.N * h->g.D * sizeof(float), cudaMemcpyDeviceToDevice,
                           as_stream(stream)));
  ASH_CUDA(enqueue_tc_coeff(h, as_stream(stream)));
  return ASH_OK;
}

ash_status ash_get_coefficients(const ash_hologram* h, float* coeff, void* stream) {
  if (!h || !coeff) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  ASH_CUDA(cudaMemcpyAsync(coeff, h->coeff, (size_t)h->g.N * h->g.D * sizeof(float), cudaMemcpyDeviceToDevice,
                           as_stream(stream)));
  return ASH_OK;
}

ash_status ash_set_amplitude(ash_hologram* h, const float* amp, void* stream) {
  if (!h || !amp) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = as_stream(stream);
  k_amp_image<<<h->g.T, h->g.NT, 0, s>>>(h->g, amp, h->amp_img);
  ASH_CUDA(cudaGetLastError());
  k_sum_sq<<<1, 1024, 0, s>>>(amp, (size_t)h->g.nx * h->g.ny, h->sum_a2);
  ASH_CUDA(cudaGetLastError());
  return ASH_OK;
}

ash_status ash_forward(ash_hologram* h, const float* phase, float* E, void* stream) {
  if (!h || !phase || !E) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  return enqueue_forward(h, kSrcPhase, phase, nullptr, reinterpret_cast<float2*>(E), as_stream(stream));
}

ash_status ash_forward_coeff(ash_hologram* h, const float* coeff, const float* phase, float* E, void* stream) {
  if (!h || !coeff || !phase || !E) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = as_stream(stream);
  ASH_CUDA(cudaMemcpyAsync(h->coeff, coeff, (size_t)h->g.N * h->g.D * sizeof(float), cudaMemcpyDeviceToDevice, s));
  ASH_CUDA(enqueue_tc_coeff(h, s));
  return enqueue_forward(h, kSrcPhase, phase, nullptr, reinterpret_cast<float2*>(E), s);
}

ash_status ash_spot_loss(const float* E, const float* t, int N, float* loss, float* grad_E, void* stream) {
  if (!E || !t || (!loss && !grad_E)) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (N < 1 || N > (1 << 20)) return set_error(ASH_ERR_INVALID_ARG, "N=%d outside [1, 2^20]", N);
  if ((reinterpret_cast<uintptr_t>(E) & 7) || (reinterpret_cast<uintptr_t>(grad_E) & 7))
    return set_error(ASH_ERR_INVALID_ARG, "complex buffers must be 8-byte aligned");
  k_spot_loss<<<1, 1024, 0, as_stream(stream)>>>(reinterpret_cast<const float2*>(E), t, N, loss,
                                                 reinterpret_cast<float2*>(grad_E));
  ASH_CUDA(cudaGetLastError());
  return ASH_OK;
}

ash_status ash_forward_field(ash_hologram* h, const float* field, float* E, void* stream) {
  if (!h || !field || !E) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(field) & 7) || (reinterpret_cast<uintptr_t>(E) & 7))
    return set_error(ASH_ERR_INVALID_ARG, "complex buffers must be 8-byte aligned");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  return enqueue_forward(h, kSrcField, nullptr, reinterpret_cast<const float2*>(field), reinterpret_cast<float2*>(E),
                         as_stream(stream));
}




ash_status ash_adjoint(ash_hologram* h, const float* y, float* g, float* phase_out, void* stream) {
  if (!h || !y) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (!g && !phase_out) return set_error(ASH_ERR_INVALID_ARG, "need g or phase_out");
  if ((reinterpret_cast<uintptr_t>(y) & 7) || (reinterpret_cast<uintptr_t>(g) & 7))
    return set_error(ASH_ERR_INVALID_ARG, "complex buffers must be 8-byte aligned");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  int epi = (g ? kEpiField : 0) | (phase_out ? kEpiPhase : 0);
  return enqueue_adjoint(h, reinterpret_cast<const float2*>(y), reinterpret_cast<float2*>(g), phase_out, nullptr,
                         nullptr, epi, as_stream(stream));
}

ash_status ash_wgs_iterate(ash_hologram* h, float* phase, float* w, const float* target, int iters, float* E_out,
                           float* metrics_out, void* stream) {
  if (!h || !phase || !w || !target) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (iters < 0 || iters > 1000000) return set_error(ASH_ERR_INVALID_ARG, "iters=%d outside [0, 1e6]", iters);
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = as_stream(stream);
  const size_t M = (size_t)h->g.nx * h->g.ny;
  const size_t N = (size_t)h->g.N;
  ASH_CUDA(cudaMemcpyAsync(h->wgs_phase, phase, M * 4, cudaMemcpyDeviceToDevice, s));
  ASH_CUDA(cudaMemcpyAsync(h->wgs_w, w, N * 4, cudaMemcpyDeviceToDevice, s));
  ASH_CUDA(cudaMemcpyAsync(h->wgs_T, target, N * 4, cudaMemcpyDeviceToDevice, s));
  if (iters >= 2) {
    cudaGraphExec_t exec = nullptr;
    ash_status st = cached_graph(h, iters, enqueue_wgs_body, iters, &exec);
    if (st != ASH_OK) return st;
    ASH_CUDA(cudaGraphLaunch(exec, s));
  } else {
    ash_status st = enqueue_wgs_body(h, iters, s);
    if (st != ASH_OK) return st;
  }
  ASH_CUDA(cudaMemcpyAsync(phase, h->wgs_phase, M * 4, cudaMemcpyDeviceToDevice, s));
  ASH_CUDA(cudaMemcpyAsync(w, h->wgs_w, N * 4, cudaMemcpyDeviceToDevice, s));
  if (E_out) ASH_CUDA(cudaMemcpyAsync(E_out, h->wgs_E, N * 8, cudaMemcpyDeviceToDevice, s));
  if (metrics_out) ASH_CUDA(cudaMemcpyAsync(metrics_out, h->wgs_metrics, 16, cudaMemcpyDeviceToDevice, s));
  return ASH_OK;
}

ash_status ash_grad(ash_hologram* h, const float* phase, const float* grad_E, float* dphase, float* dcoeff,
                    void* stream) {
  if (!h || !phase || !grad_E) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (!dphase && !dcoeff) return set_error(ASH_ERR_INVALID_ARG, "need dphase or dcoeff");
  if (reinterpret_cast<uintptr_t>(grad_E) & 7) return set_error(ASH_ERR_INVALID_ARG, "grad_E must be 8-byte aligned");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = as_stream(stream);
  const float2* gE = reinterpret_cast<const float2*>(grad_E);
  if (dphase) {
    ash_status st = enqueue_adjoint(h, gE, nullptr, nullptr, phase, dphase, kEpiGradPhase, s);
    if (st != ASH_OK) return st;
  }
  if (dcoeff && use_tc_grad(h)) {
    ASH_CUDA(enqueue_tc_gradc(h, phase, gE, dcoeff, s));
  } else if (dcoeff) {
    if (!h->dz) return set_error(ASH_ERR_DEVICE, "FMA-pipe moments without their basis image");
    GradCParams p{};
    p.v = view_of(h);
    p.phase = phase;
    p.gradE = gE;
    p.partial = h->gradc_partial;
    cudaError_t e = launch_gradc(h->g.D, p, dim3(h->gradc_gx, h->gradc_gy), s);
    if (e != cudaSuccess) return cuda_fail(e, "gradc kernel launch");
    const int cols = h->g.N * h->g.D;
    k_col_reduce<<<(cols + 31) / 32, dim3(32, 32), 0, s>>>(h->gradc_partial, h->gradc_gx, cols, dcoeff);
    ASH_CUDA(cudaGetLastError());
  }
  return ASH_OK;
}

ash_status ash_hologram_launch_info(const ash_hologram* h, int* out) {
  if (!h || !out) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  out[0] = h->sched.G;
  out[1] = h->li.fwd_ctas_per_sm;
  out[2] = h->li.adj_ctas_per_sm;
  out[3] = h->tc_ok ? h->tadj.G : 0;
  out[4] = h->tc_ok ? h->tfwd.G : 0;
  out[5] = (h->split_tiles ? 1 : 0) | (h->tadj_split ? 2 : 0) | (h->tfwd_split ? 4 : 0) |
           (h->tfwd_nfull >= 0 ? 8 : 0);
  out[6] = (use_tc_adj(h) ? 2 : 1) | (use_tc_fwd(h) ? 4 : 0) | (use_tc_grad(h) ? 8 : 0);
  out[7] = h->g.P;
  return ASH_OK;
}

ash_status ash_set_kernel_variant(ash_hologram* h, int variant) {
  if (!h || variant < 0 || variant > 2) return set_error(ASH_ERR_INVALID_ARG, "variant must be 0, 1 or 2");
  if (variant == 2 && !h->tc_ok)
    return set_error(ASH_ERR_UNSUPPORTED, "tensor-core kernels need D <= %d (D = %d)", kTcMaxModes, h->g.D);
  h->variant = variant;
  clear_graphs(h);
  if (needs_fma_image(h)) return ensure_fma_image(h);
  return ASH_OK;
}

ash_status ash_wgs_set_options(ash_hologram* h, float feedback, int fix_phase) {
  if (!h) return set_error(ASH_ERR_INVALID_ARG, "handle is NULL");
  if (!(feedback >= 0.0f && feedback <= 16.0f)) return set_error(ASH_ERR_INVALID_ARG, "feedback outside [0, 16]");
  if (fix_phase != 0 && fix_phase != 1) return set_error(ASH_ERR_INVALID_ARG, "fix_phase must be 0 or 1");
  h->wgs_feedback = feedback;
  h->wgs_fix = fix_phase != 0;
  clear_graphs(h);   // the graphs hold the old options
  return ASH_OK;
}

int ash_graph_kernels(const ash_hologram* h, int key) {
  if (!h) return -1;
  auto it = h->graphs.find(key);
  return it == h->graphs.end() ? -1 : it->second.kernels;
}

int ash_wgs_launches(const ash_hologram* h, int iters) {
  if (!h || iters < 0) return -1;
  // forward: tensor-core (nearfield image unless fused, kernel, reduce if
  // split) or FMA (kernel, reduction); adjoint: kernel (+ fix-up)
  const bool fused = wgs_fused_field(h);
  const int fwd_first = use_tc_fwd(h) ? 2 + (h->tfwd_split ? 1 : 0) : 2;
  const int fwd = use_tc_fwd(h) ? (fused ? 1 : 2) + (h->tfwd_split ? 1 : 0) : 2;
  const int adj = use_tc_adj(h) ? 1 + (h->tadj_split ? 1 : 0) : 1 + (h->split_tiles ? 1 : 0);
  return fwd_first + iters * (1 + adj + fwd) + 1;   // + metrics
}

ash_status ash_profile(ash_hologram* h, const float* phase, const float* y, float* ms_out, void* stream) {
  if (!h || !phase || !y || !ms_out) return set_error(ASH_ERR_INVALID_ARG, "NULL argument");
  if (reinterpret_cast<uintptr_t>(y) & 7) return set_error(ASH_ERR_INVALID_ARG, "y must be 8-byte aligned");
  if (injected_failure()) return set_error(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = as_stream(stream);
  if (needs_fma_image(h) && !h->dz) return set_error(ASH_ERR_DEVICE, "FMA-pipe kernels without their basis image");
  cudaEvent_t ev[12];
  for (int q = 0; q < 12; ++q) ASH_CUDA(cudaEventCreate(&ev[q]));
  const float2* y2 = reinterpret_cast<const float2*>(y);
  ash_status st = ASH_OK;
  cudaError_t e = cudaSuccess;
  // forward kernel, then its reduction
  FwdParams fp{};
  fp.v = view_of(h);
  fp.sched = h->sched;
  fp.phase = phase;
  fp.source = kSrcPhase;
  fp.partial = h->partial;
  const int cols = 2 * h->g.N;
  const bool tc = use_tc_fwd(h), tca = use_tc_adj(h);
  const TcFwdParams tf = tc_fwd_params(h, h->E);
  if (tc) e = tc_field_img(h->g, h->amp_img, phase, nullptr, h->fimg, s);
  cudaEventRecord(ev[0], s);
  if (e == cudaSuccess) e = tc ? tc_launch_forward(h->tc_na, tf, h->tfwd.G, s) : launch_forward(h->g.D, fp, h->sched.G, s);
  cudaEventRecord(ev[1], s);
  if (e == cudaSuccess) {
    cudaEventRecord(ev[2], s);
    if (!tc) {
      k_col_reduce<<<(cols + 31) / 32, dim3(32, 32), 0, s>>>(h->partial, h->fwd_rows, cols, reinterpret_cast<float*>(h->E));
      e = cudaGetLastError();
    } else if (h->tfwd_split) {
      e = tc_launch_forward_reduce(tf, s);
    }
    cudaEventRecord(ev[3], s);
  }
  // adjoint kernel (phase epilogue), then the fix-up
  AdjParams ap{};
  ap.v = view_of(h);
  ap.sched = h->sched;
  ap.split = h->split;
  ap.y = y2;
  ap.out.phase_out = h->wgs_phase;
  ap.out.epilogue = kEpiPhase;
  const TcAdjParams tp = tc_adj_params(h, y2, ap.out);
  if (e == cudaSuccess) {
    cudaEventRecord(ev[4], s);
    e = tca ? tc_launch_adjoint(h->tc_na, tp, h->tadj.G, s) : launch_adjoint(h->g.D, ap, h->sched.G, s);
    cudaEventRecord(ev[5], s);
  }
  if (e == cudaSuccess) {
    cudaEventRecord(ev[6], s);
    if (tca && h->tadj_split) {
      e = tc_launch_adjoint_fixup(tp, h->tadj_nsplit, s);
    } else if (!tca && h->split_tiles) {
      k_adjoint_fixup<<<h->g.T, h->g.NT, 0, s>>>(ap);
      e = cudaGetLastError();
    }
    cudaEventRecord(ev[7], s);
  }
  if (e == cudaSuccess) {
    cudaEventRecord(ev[8], s);
    k_wgs_update<<<1, 1024, 0, s>>>(h->E, h->wgs_w, reinterpret_cast<const float*>(h->wgs_T), h->y, h->g.N, 1.0f,
                                    nullptr, nullptr);
    e = cudaGetLastError();
    cudaEventRecord(ev[9], s);
  }
  if (e == cudaSuccess) {
    GradCParams gp{};
    gp.v = view_of(h);
    gp.phase = phase;
    gp.gradE = y2;
    gp.partial = h->gradc_partial;
    cudaEventRecord(ev[10], s);
    e = use_tc_grad(h) ? tc_launch_gradc(tc_grad_params(h, y2, h->gradc_partial), h->tgrad_split, s)
                       : launch_gradc(h->g.D, gp, dim3(h->gradc_gx, h->gradc_gy), s);
    cudaEventRecord(ev[11], s);
  }
  if (e != cudaSuccess) st = cuda_fail(e, "profile launch");
  cudaError_t se = cudaStreamSynchronize(s);
  if (st == ASH_OK && se != cudaSuccess) st = cuda_fail(se, "profile synchronise");
  if (st == ASH_OK) {
    for (int q = 0; q < 6; ++q) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[2 * q], ev[2 * q + 1]);
      ms_out[q] = ms;
    }
  }
  for (int q = 0; q < 12; ++q) cudaEventDestroy(ev[q]);
  return st;
}

ash_status ash_hologram_check(ash_hologram* h, void* stream) {
  if (!h) return set_error(ASH_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t s = as_stream(stream);
  unsigned word = 0;
  ASH_CUDA(cudaMemcpyAsync(&word, h->err_word, sizeof word, cudaMemcpyDeviceToHost, s));
  ASH_CUDA(cudaStreamSynchronize(s));
  if (word) {
    ASH_CUDA(cudaMemsetAsync(h->err_word, 0, sizeof word, s));
    ASH_CUDA(cudaStreamSynchronize(s));
    if (word & kErrTimeout)
      return set_error(ASH_ERR_TIMEOUT, "a bounded wait gave up (device error word 0x%x)", word);
    return set_error(ASH_ERR_DEVICE, "device error word 0x%x", word);
  }
  return ASH_OK;
}

ash_status ash_debug_wait_timeout(ash_hologram* h, unsigned polls, void* stream) {
  if (!h) return set_error(ASH_ERR_INVALID_ARG, "handle is NULL");
  if (polls < 1 || polls > (1u << 20)) return set_error(ASH_ERR_INVALID_ARG, "polls outside [1, 2^20]");
  k_debug_wait<<<1, 32, 0, as_stream(stream)>>>(polls, h->err_word);
  ASH_CUDA(cudaGetLastError());
  return ASH_OK;
}

}  // extern "C"
