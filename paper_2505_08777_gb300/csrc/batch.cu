// Batched uneven form: many holograms of different grid sizes, spot counts
// and mode counts solved together, one persistent launch per phase of the
// weighted-GS iteration, the whole loop captured in one CUDA graph.
//
// Work units are (hologram, tile, spot) triples, hologram-major then
// tile-major; the G CTAs of a launch get equal contiguous ranges of the
// global unit sequence, so small and large holograms share the GPU without
// tail effects. Each tile is dispatched on its hologram's D to the same
// specialised tile code the single-hologram kernels use. Tiles split between
// CTAs are finished by a fix-up pass in a fixed CTA order (deterministic).
//
// When every hologram has the tensor-core operand images (same K-atom count),
// the batch runs the tensor-core transforms instead: persistent CTAs walk
// their equal slice of the concatenated (hologram, group, spot chunk) /
// (hologram, spot block, pixel chunk) units hologram by hologram, with the
// same per-range code as the single-hologram kernels; each hologram sees the
// CTAs that meet it as its own local CTAs, with its own boundary table,
// split slots and fix-up / reduction work.
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "aux_kernels.cuh"
#include "handle.h"
#include "tc_launch.h"
#include "transform_kernels.cuh"

namespace {

using namespace ash;

constexpr int kBatchP = 8;                 // pixels per thread (D <= 12)
constexpr int kBatchNT = kTilePix / kBatchP;
constexpr int kBatchNW = kBatchNT / 32;
constexpr int kBatchMaxD = 12;
// Members whose N * M reaches this many terms run standalone inside the
// batch's graph (their own tuned single-hologram kernels); smaller ones share
// the persistent launches, where one launch per phase replaces one per
// hologram.
constexpr long long kBatchSoloTerms = 1LL << 22;
constexpr int kGridFactorMax = 4;          // split scratch sized for 4x the resident CTAs

struct BatchHolo {
  HoloView v;
  long long unit0;       // first global work unit
  int tile0;             // first global tile
  float* partial;        // forward partial rows [T * NW][2N]
  float2* E;
  float2* y;
  float* w;
  const float* T;
  float* phase;
  float* metrics;
  const double* sum_a2;
};

struct BatchParams {
  const BatchHolo* holos;
  int count;
  Schedule sched;
  float2* split;
};

__device__ __forceinline__ int holo_of_unit(const BatchHolo* __restrict__ hs, int count, long long u) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (hs[mid].unit0 <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int holo_of_tile(const BatchHolo* __restrict__ hs, int count, int gt) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (hs[mid].tile0 <= gt) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr size_t batch_fwd_smem() { return fwd_smem_bytes(kBatchMaxD); }
constexpr size_t batch_adj_smem() { return adj_smem_bytes(kBatchMaxD); }

#define ASH_D_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

// Out-of-line per-D tile bodies: each is register-allocated on its own, so
// the batched kernels cost about as many registers as the single-hologram
// kernel of the largest D instead of the sum of all inlined cases.
template <int D>
__device__ __noinline__ void batch_forward_tile(const BatchHolo* __restrict__ H, int tile, int sb, int se,
                                                float* sC, float2* sRot) {
  const HoloView v = H->v;
  forward_tile<D, kBatchP>(v, kSrcPhase, H->phase, nullptr, tile, sb, se,
                           H->partial + (size_t)tile * kBatchNW * 2 * v.g.N, sC, sRot);
}

template <int D>
__device__ __noinline__ void batch_adjoint_tile(const BatchHolo* __restrict__ H, int tile, int sb, int se,
                                                float2* slot, float* sC, float4* sY) {
  const HoloView v = H->v;
  float2 re2[kBatchP / 2], im2[kBatchP / 2];
  adjoint_tile<D, kBatchP>(v, H->y, tile, sb, se, re2, im2, sC, sY);
  AdjOut out{};
  out.phase_out = H->phase;
  out.epilogue = kEpiPhase;
  adjoint_finish<kBatchP>(v, out, tile, sb == 0 && se == v.g.N, slot, re2, im2);
}

// DMAX: largest mode count of the batch; only cases up to DMAX are reachable,
// so the kernel's register count is that of the largest case present.
template <int DMAX>
__global__ void ASH_BOUNDS(kBatchP) k_batch_forward(const BatchParams bp) {
  extern __shared__ float4 smem4[];
  float* sC = reinterpret_cast<float*>(smem4);
  float2* sRot = reinterpret_cast<float2*>(sC + kSpotChunk * cpair_stride(kBatchMaxD));
  const long long u0 = bp.sched.begin(blockIdx.x), u1 = bp.sched.begin(blockIdx.x + 1);
  long long u = u0;
  while (u < u1) {
    const BatchHolo* H = bp.holos + holo_of_unit(bp.holos, bp.count, u);
    const HoloView v = H->v;
    const int N = v.g.N;
    const int tile = (int)((u - H->unit0) / N);
    const long long ts = H->unit0 + (long long)tile * N;
    const long long ue = min(u1, ts + N);
    const int sb = (int)(u - ts), se = (int)(ue - ts);
    switch (v.g.D) {
#define FWD_CASE(DD) \
  case DD: if constexpr (DD <= DMAX) batch_forward_tile<DD>(H, tile, sb, se, sC, sRot); break;
      ASH_D_CASES(FWD_CASE)
#undef FWD_CASE
      default: break;
    }
    u = ue;
  }
}

template <int DMAX>
__global__ void ASH_BOUNDS(kBatchP) k_batch_adjoint(const BatchParams bp) {
  extern __shared__ float4 smem4[];
  float* sC = reinterpret_cast<float*>(smem4);
  float4* sY = reinterpret_cast<float4*>(sC + kSpotChunk * cpair_stride(kBatchMaxD));
  const long long u0 = bp.sched.begin(blockIdx.x), u1 = bp.sched.begin(blockIdx.x + 1);
  long long u = u0;
  while (u < u1) {
    const BatchHolo* H = bp.holos + holo_of_unit(bp.holos, bp.count, u);
    const HoloView v = H->v;
    const int N = v.g.N;
    const int tile = (int)((u - H->unit0) / N);
    const long long ts = H->unit0 + (long long)tile * N;
    const long long ue = min(u1, ts + N);
    const int sb = (int)(u - ts), se = (int)(ue - ts);
    float2* slot = bp.split + ((size_t)blockIdx.x * 2 + (u == u0 ? 0 : 1)) * kTilePix;
    switch (v.g.D) {
#define ADJ_CASE(DD) \
  case DD: if constexpr (DD <= DMAX) batch_adjoint_tile<DD>(H, tile, sb, se, slot, sC, sY); break;
      ASH_D_CASES(ADJ_CASE)
#undef ADJ_CASE
      default: break;
    }
    u = ue;
  }
}

// One CTA per global tile; tiles owned by a single CTA return at once.
__global__ void k_batch_fixup(const BatchParams bp) {
  const BatchHolo* H = bp.holos + holo_of_tile(bp.holos, bp.count, blockIdx.x);
  const int tile = blockIdx.x - H->tile0;
  const int N = H->v.g.N;
  const long long u_lo = H->unit0 + (long long)tile * N, u_hi = u_lo + N - 1;
  const int b_lo = bp.sched.owner(u_lo), b_hi = bp.sched.owner(u_hi);
  if (b_lo == b_hi) return;
  AdjOut out{};
  out.phase_out = H->phase;
  out.epilogue = kEpiPhase;
  fixup_tile_body(H->v, out, bp.split, bp.sched, tile, u_lo, b_lo, b_hi);
}

// grid (max columns / 32, count), block (32, 32)
__global__ void k_batch_reduce(const BatchParams bp) {
  const BatchHolo* H = bp.holos + blockIdx.y;
  const int cols = 2 * H->v.g.N;
  if ((int)blockIdx.x * 32 >= cols) return;
  col_reduce_body(H->partial, H->v.g.T * kBatchNW, cols, reinterpret_cast<float*>(H->E), blockIdx.x);
}

__global__ void __launch_bounds__(1024) k_batch_update(const BatchParams bp) {
  const BatchHolo* H = bp.holos + blockIdx.x;
  wgs_update_body(H->E, H->w, H->T, H->y, H->v.g.N);
}

__global__ void __launch_bounds__(1024) k_batch_metrics(const BatchParams bp) {
  const BatchHolo* H = bp.holos + blockIdx.x;
  metrics_body(H->E, H->T, H->v.g.N, H->sum_a2, (double)H->v.g.nx * H->v.g.ny, H->metrics);
}

ash_status fail(ash_status st, const std::string& msg) {
  record_error(msg.c_str());
  return st;
}

// Max-D classes with their own kernel instantiations.
constexpr int kDClasses[] = {4, 6, 8, 10, 11, 12};
using BatchKernel = void (*)(BatchParams);

BatchKernel fwd_kernel(int dmax) {
  switch (dmax) {
    case 4: return k_batch_forward<4>;
    case 6: return k_batch_forward<6>;
    case 8: return k_batch_forward<8>;
    case 10: return k_batch_forward<10>;
    case 11: return k_batch_forward<11>;
    default: return k_batch_forward<12>;
  }
}

BatchKernel adj_kernel(int dmax) {
  switch (dmax) {
    case 4: return k_batch_adjoint<4>;
    case 6: return k_batch_adjoint<6>;
    case 8: return k_batch_adjoint<8>;
    case 10: return k_batch_adjoint<10>;
    case 11: return k_batch_adjoint<11>;
    default: return k_batch_adjoint<12>;
  }
}

#define BCUDA(call)                                            \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return status_cuda(e_, #call);      \
  } while (0)

}  // namespace

struct ash_batch {
  // members with N*M >= solo_terms run standalone (their own single-hologram
  // kernels, in the batch's graph); the others share the persistent batched
  // launches below, whose fields all refer to that group only
  int members = 0;
  int device = 0, sms = 0;
  std::vector<ash_hologram*> all;    // every member, in the caller's order
  std::vector<ash_hologram*> solo;   // the standalone members
  std::vector<int> group_idx;        // member index of each persistent-group hologram
  long long solo_terms = 0;
  int count = 0;                     // members in the persistent group
  std::vector<ash_hologram*> holos;
  std::vector<BatchHolo> host;
  BatchHolo* dev = nullptr;
  long long U = 0;
  int total_tiles = 0;
  int max_cols = 0;
  int slots = 0;           // resident CTAs on the device
  int dclass = 12;         // kernel instantiation: max D of the batch, rounded up to a class
  BatchKernel fwd = nullptr, adj = nullptr;
  int G = 0;               // CTAs of the transform launches
  bool split = false;
  float2* split_buf = nullptr;
  cudaStream_t capture = nullptr;
  std::map<int, cudaGraphExec_t> graphs;
  std::map<int, int> graph_kernels;   // kernel nodes of each cached graph
  // tensor-core path
  int variant = 0;         // 0 auto, 1 FMA-pipe kernels, 2 tensor-core kernels
  bool tc_ok = false;      // every hologram has tensor-core images with the same K-atom count
  int tc_na = 0;
  int tc_slots = 0;        // resident CTAs of the tensor-core adjoint
  int tc_fwd_per_sm = 0, tc_adj_per_sm = 0;
  TcAdjParams* d_adj = nullptr;
  TcFwdParams* d_fwd = nullptr;
  long long* d_hu0 = nullptr;      // [2][count + 1] unit offsets: adjoint, forward
  int* d_g0 = nullptr;             // [2][count] first CTA meeting each hologram
  long long* d_begin = nullptr;    // per-hologram CTA boundary tables
  float2* d_tsplit = nullptr;      // per-hologram split slots
  int4* d_lists = nullptr;         // adjoint fix-up list, then forward reduction list
  TcFieldDesc* d_field = nullptr;
  int* d_tiles0 = nullptr;
  TcBatchSched bs_adj{}, bs_fwd{};
  int n_fix = 0, n_red = 0;
  size_t cap_begin = 0, cap_split = 0, cap_fix = 0;
  bool use_tc() const { return tc_ok && variant != 1; }
};

namespace {

// CTA boundary tables, split slots and work lists of the tensor-core
// launches for the current grid (adjoint grid G, forward grid scaled by the
// two kernels' resident CTAs per SM).
ash_status build_tc(ash_batch* b) {
  const int count = b->count;
  std::vector<long long> hu0(2 * (count + 1)), begins;
  std::vector<int> g0(2 * count);
  std::vector<int4> fix, red;   // (hologram, group or block, first CTA, last CTA) in local CTA numbers
  std::vector<TcAdjParams> adj(count);
  std::vector<TcFwdParams> fwd(count);
  size_t split_off = 0;
  for (int x = 0; x < 2; ++x) {   // 0 adjoint, 1 forward
    long long* off = &hu0[(size_t)x * (count + 1)];
    off[0] = 0;
    for (int h = 0; h < count; ++h) {
      const Geometry& g = b->holos[h]->g;
      const long long W = x == 0 ? (long long)g.T * kTcGroupsPerTile * ((g.N + kTcChunk - 1) / kTcChunk)
                                 : (long long)((g.N + kTcRows - 1) / kTcRows) * g.T * kTcChunksPerTile;
      off[h + 1] = off[h] + W;
    }
    const long long U = off[count];
    long long Gl = x == 0 ? b->G : ((long long)b->G * b->tc_fwd_per_sm) / (b->tc_adj_per_sm > 0 ? b->tc_adj_per_sm : 1);
    if (Gl < 1) Gl = 1;
    if (Gl > U) Gl = U;
    const int G = (int)Gl;
    TcBatchSched& bs = x == 0 ? b->bs_adj : b->bs_fwd;
    bs.count = count;
    bs.U = U;
    bs.G = G;
    auto owner = [&](long long u) {
      int lo = 0, hi = G - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (bs.begin(mid) <= u) lo = mid;
        else hi = mid - 1;
      }
      return lo;
    };
    for (int h = 0; h < count; ++h) {
      const ash_hologram* H = b->holos[h];
      const Geometry& g = H->g;
      const long long Uh = off[h], Wh = off[h + 1] - off[h];
      const int ga = owner(Uh), gb = owner(Uh + Wh - 1), Gh = gb - ga + 1;
      g0[(size_t)x * count + h] = ga;
      const size_t tab = begins.size();
      for (int k = 0; k <= Gh; ++k) {
        const long long v = bs.begin(ga + k) - Uh;
        begins.push_back(v < 0 ? 0 : (v > Wh ? Wh : v));
      }
      const size_t so = split_off;
      split_off += (size_t)Gh * 2 * kTcRows;
      if (x == 0) {
        const int nch = (g.N + kTcChunk - 1) / kTcChunk;
        for (int k = 1; k < Gh; ++k) {
          const long long u = begins[tab + k];
          if (u % nch == 0) continue;
          const int grp = (int)(u / nch);
          if (fix.empty() || fix.back().x != h || fix.back().y != grp) {
            const long long ulo = (long long)grp * nch;
            fix.push_back(make_int4(h, grp, tc_owner(begins.data() + tab, Gh, ulo),
                                    tc_owner(begins.data() + tab, Gh, ulo + nch - 1)));
          }
        }
        TcAdjParams& p = adj[h];
        p.g = g;
        p.zs = H->zs;
        p.czs = H->czs;
        p.rot = H->rot;
        p.y = H->y;
        p.amp_img = H->amp_img;
        p.out.phase_out = H->wgs_phase;
        p.out.epilogue = kEpiPhase | kEpiFimg;
        p.fimg = H->fimg;
        p.begin = reinterpret_cast<const long long*>(tab);    // offsets, rebased below
        p.G = Gh;
        p.split = reinterpret_cast<float2*>(so);
        p.err = H->err_word;
      } else {
        TcFwdParams& p = fwd[h];
        p.g = g;
        p.zs = H->zs;
        p.czs = H->czs;
        p.rot = H->rot;
        p.fimg = H->fimg;
        p.sched.nb = (g.N + kTcRows - 1) / kTcRows;
        p.sched.nq = g.T * kTcChunksPerTile;
        p.sched.G = Gh;
        p.rep = tc_fwd_rep(g.N);
        p.begin = reinterpret_cast<const long long*>(tab);
        p.E = H->wgs_E;
        p.part = reinterpret_cast<float2*>(so);
        p.err = H->err_word;
        for (int blk = 0; blk < p.sched.nb; ++blk) {
          const long long ulo = (long long)blk * p.sched.nq;
          red.push_back(make_int4(h, blk, tc_owner(begins.data() + tab, Gh, ulo),
                                  tc_owner(begins.data() + tab, Gh, ulo + p.sched.nq - 1)));
        }
      }
    }
  }
  if (begins.size() > b->cap_begin || split_off > b->cap_split || fix.size() + red.size() > b->cap_fix)
    return fail(ASH_ERR_INVALID_ARG, "batch tensor-core tables exceed their capacity");
  for (auto& p : adj) {
    p.begin = b->d_begin + reinterpret_cast<size_t>(p.begin);
    p.split = b->d_tsplit + reinterpret_cast<size_t>(p.split);
  }
  for (auto& p : fwd) {
    p.begin = b->d_begin + reinterpret_cast<size_t>(p.begin);
    p.part = b->d_tsplit + reinterpret_cast<size_t>(p.part);
  }
  b->n_fix = (int)fix.size();
  b->n_red = (int)red.size();
  std::vector<int4> lists(fix);
  lists.insert(lists.end(), red.begin(), red.end());
  b->bs_adj.hu0 = b->d_hu0;
  b->bs_adj.g0 = b->d_g0;
  b->bs_fwd.hu0 = b->d_hu0 + (count + 1);
  b->bs_fwd.g0 = b->d_g0 + count;
  cudaError_t e;
  if ((e = cudaMemcpy(b->d_hu0, hu0.data(), hu0.size() * sizeof(long long), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_g0, g0.data(), g0.size() * sizeof(int), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_begin, begins.data(), begins.size() * sizeof(long long), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_adj, adj.data(), adj.size() * sizeof(TcAdjParams), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_fwd, fwd.data(), fwd.size() * sizeof(TcFwdParams), cudaMemcpyHostToDevice)) ||
      (!lists.empty() &&
       (e = cudaMemcpy(b->d_lists, lists.data(), lists.size() * sizeof(int4), cudaMemcpyHostToDevice))))
    return status_cuda(e, "batch tensor-core tables");
  return ASH_OK;
}

ash_status set_grid(ash_batch* b, int G) {
  if (b->count == 0) return ASH_OK;   // every member is standalone
  const int slots = b->use_tc() ? b->tc_slots : b->slots;
  if (G < 1) G = 1;
  if (G > kGridFactorMax * slots) G = kGridFactorMax * slots;
  if (!b->use_tc() && (long long)G > b->U) G = (int)b->U;
  if (G != b->G) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->graph_kernels.clear();
  }
  b->G = G;
  Schedule s{b->U, G};
  b->split = false;
  // a tile is split iff some CTA boundary falls inside it
  for (int g = 1; g < G && !b->split; ++g) {
    const long long u = s.begin(g);
    for (const BatchHolo& h : b->host) {
      const long long end = h.unit0 + (long long)h.v.g.T * h.v.g.N;
      if (u >= h.unit0 && u < end) {
        if ((u - h.unit0) % h.v.g.N != 0) b->split = true;
        break;
      }
    }
  }
  if (b->use_tc()) return build_tc(b);
  return ASH_OK;
}

BatchParams params_of(const ash_batch* b) {
  BatchParams p{};
  p.holos = b->dev;
  p.count = b->count;
  p.sched = Schedule{b->U, b->G};
  p.split = b->split_buf;
  return p;
}

ash_status enqueue_batch_forward(ash_batch* b, cudaStream_t s) {
  const BatchParams p = params_of(b);
  b->fwd<<<b->G, kBatchNT, batch_fwd_smem(), s>>>(p);
  BCUDA(cudaGetLastError());
  k_batch_reduce<<<dim3((b->max_cols + 31) / 32, b->count), dim3(32, 32), 0, s>>>(p);
  BCUDA(cudaGetLastError());
  return ASH_OK;
}

ash_status enqueue_batch_adjoint(ash_batch* b, cudaStream_t s) {
  const BatchParams p = params_of(b);
  b->adj<<<b->G, kBatchNT, batch_adj_smem(), s>>>(p);
  BCUDA(cudaGetLastError());
  if (b->split) {
    k_batch_fixup<<<b->total_tiles, kBatchNT, 0, s>>>(p);
    BCUDA(cudaGetLastError());
  }
  return ASH_OK;
}

ash_status enqueue_tc_forward(ash_batch* b, cudaStream_t s) {
  BCUDA(tc_launch_forward_batch(b->tc_na, b->d_fwd, b->bs_fwd, s));
  BCUDA(tc_launch_forward_reduce_batch(b->d_fwd, b->d_lists + b->n_fix, b->n_red, s));
  return ASH_OK;
}

ash_status enqueue_tc_adjoint(ash_batch* b, cudaStream_t s) {
  BCUDA(tc_launch_adjoint_batch(b->tc_na, b->d_adj, b->bs_adj, s));
  BCUDA(tc_launch_adjoint_fixup_batch(b->d_adj, b->d_lists, b->n_fix, s));
  return ASH_OK;
}

// Tensor-core loop: the first forward converts the phases; every adjoint
// also writes the next forward's nearfield images.
ash_status enqueue_tc_body(ash_batch* b, int iters, cudaStream_t s) {
  const BatchParams p = params_of(b);
  ash_status st;
  BCUDA(tc_field_img_batch(b->d_field, b->d_tiles0, b->count, b->total_tiles, s));
  if ((st = enqueue_tc_forward(b, s)) != ASH_OK) return st;
  for (int it = 0; it < iters; ++it) {
    k_batch_update<<<b->count, 1024, 0, s>>>(p);
    BCUDA(cudaGetLastError());
    if ((st = enqueue_tc_adjoint(b, s)) != ASH_OK) return st;
    if ((st = enqueue_tc_forward(b, s)) != ASH_OK) return st;
  }
  k_batch_metrics<<<b->count, 1024, 0, s>>>(p);
  BCUDA(cudaGetLastError());
  return ASH_OK;
}

ash_status enqueue_batch_body(ash_batch* b, int iters, cudaStream_t s) {
  if (b->use_tc()) return enqueue_tc_body(b, iters, s);
  const BatchParams p = params_of(b);
  ash_status st;
  for (int it = 0; it < iters; ++it) {
    if ((st = enqueue_batch_forward(b, s)) != ASH_OK) return st;
    k_batch_update<<<b->count, 1024, 0, s>>>(p);
    BCUDA(cudaGetLastError());
    if ((st = enqueue_batch_adjoint(b, s)) != ASH_OK) return st;
  }
  if ((st = enqueue_batch_forward(b, s)) != ASH_OK) return st;
  k_batch_metrics<<<b->count, 1024, 0, s>>>(p);
  BCUDA(cudaGetLastError());
  return ASH_OK;
}

// Persistent-group resources (everything but the member handles).
void release_group(ash_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
  b->graph_kernels.clear();
  if (b->dev) cudaFree(b->dev);
  if (b->split_buf) cudaFree(b->split_buf);
  for (void* q : {(void*)b->d_adj, (void*)b->d_fwd, (void*)b->d_hu0, (void*)b->d_g0, (void*)b->d_begin,
                  (void*)b->d_tsplit, (void*)b->d_lists, (void*)b->d_field, (void*)b->d_tiles0})
    if (q) cudaFree(q);
  b->dev = nullptr;
  b->split_buf = nullptr;
  b->d_adj = nullptr;
  b->d_fwd = nullptr;
  b->d_hu0 = nullptr;
  b->d_g0 = nullptr;
  b->d_begin = nullptr;
  b->d_tsplit = nullptr;
  b->d_lists = nullptr;
  b->d_field = nullptr;
  b->d_tiles0 = nullptr;
  b->solo.clear();
  b->group_idx.clear();
  b->holos.clear();
  b->host.clear();
  b->count = 0;
  b->U = 0;
  b->total_tiles = 0;
  b->max_cols = 0;
  b->G = 0;
  b->tc_ok = false;
}

void destroy_batch(ash_batch* b) {
  cudaDeviceSynchronize();
  release_group(b);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (ash_hologram* h : b->all) ash_hologram_destroy(h);
  delete b;
}

// Split the members into standalone ones (N * M >= solo_terms, or D beyond
// the persistent kernels) and the persistent group, and build the group's
// descriptor table, split scratch and tensor-core tables.
ash_status build_group(ash_batch* b, long long solo_terms, cudaStream_t s) {
  cudaDeviceSynchronize();   // the previous grouping's graphs and tables may still be in use
  release_group(b);
  b->solo_terms = solo_terms;
  for (int i = 0; i < b->members; ++i) {
    ash_hologram* h = b->all[i];
    const long long terms = (long long)h->g.N * h->g.nx * h->g.ny;
    if (terms >= solo_terms || h->g.D > kBatchMaxD) {
      b->solo.push_back(h);
      // a standalone member runs the batch's kernel family
      const ash_status st = ash_set_kernel_variant(h, b->variant == 2 && !h->tc_ok ? 0 : b->variant);
      if (st != ASH_OK) return st;
      continue;
    }
    b->group_idx.push_back(i);
    b->holos.push_back(h);
    // the persistent FMA-pipe kernels read the register-image basis
    ash_status st = ensure_fma_image(h);
    if (st != ASH_OK) return st;
    BatchHolo bh{};
    bh.v = view_of(h);
    bh.unit0 = b->U;
    bh.tile0 = b->total_tiles;
    bh.partial = h->partial;
    bh.E = h->wgs_E;
    bh.y = h->y;
    bh.w = h->wgs_w;
    bh.T = h->wgs_T;
    bh.phase = h->wgs_phase;
    bh.metrics = h->wgs_metrics;
    bh.sum_a2 = h->sum_a2;
    b->host.push_back(bh);
    b->U += (long long)h->g.T * h->g.N;
    b->total_tiles += h->g.T;
    if (2 * h->g.N > b->max_cols) b->max_cols = 2 * h->g.N;
  }
  b->count = (int)b->group_idx.size();
  if (b->count == 0) return ASH_OK;   // every member standalone: no persistent group
  const int count = b->count;
  const int sms = b->sms;
  int dmax = 1;
  for (const ash_hologram* h : b->holos) dmax = h->g.D > dmax ? h->g.D : dmax;
  for (int c : kDClasses)
    if (c >= dmax) {
      b->dclass = c;
      break;
    }
  b->fwd = fwd_kernel(b->dclass);
  b->adj = adj_kernel(b->dclass);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(b->fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_fwd_smem())) !=
      cudaSuccess)
    return status_cuda(e, "batch forward attribute");
  if ((e = cudaFuncSetAttribute(b->adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_adj_smem())) !=
      cudaSuccess)
    return status_cuda(e, "batch adjoint attribute");
  int occ_f = 0, occ_a = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, b->fwd, kBatchNT, batch_fwd_smem());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_a, b->adj, kBatchNT, batch_adj_smem());
  int occ = occ_f < occ_a ? occ_f : occ_a;
  if (occ < 1) occ = 1;
  b->slots = sms * occ;
  if ((e = cudaMalloc(&b->dev, sizeof(BatchHolo) * count)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ASH_ERR_OOM, "batch descriptor allocation");
  }
  if ((e = cudaMalloc(&b->split_buf, sizeof(float2) * (size_t)kGridFactorMax * b->slots * 2 * kTilePix)) !=
      cudaSuccess) {
    cudaGetLastError();
    return fail(ASH_ERR_OOM, "batch split scratch allocation");
  }
  if ((e = cudaMemcpyAsync(b->dev, b->host.data(), sizeof(BatchHolo) * count, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return status_cuda(e, "batch descriptor upload");
  // tensor-core path: every hologram has the operand images, one K-atom count
  b->tc_ok = true;
  for (const ash_hologram* h : b->holos)
    if (!h->tc_ok || h->tc_na != b->holos[0]->tc_na) b->tc_ok = false;
  if (b->tc_ok) {
    b->tc_na = b->holos[0]->tc_na;
    // the batch kernels' smem limits are set with the single-hologram kernels' (tc_prepare)
    if ((e = tc_batch_ctas_per_sm(b->tc_na, &b->tc_adj_per_sm, &b->tc_fwd_per_sm)) != cudaSuccess)
      return status_cuda(e, "batch tensor-core occupancy");
    b->tc_slots = sms * b->tc_adj_per_sm;
    const size_t gmax = (size_t)kGridFactorMax * b->tc_slots;
    size_t blocks = 0;
    std::vector<TcFieldDesc> fd(count);
    std::vector<int> tiles0(count);
    int t0 = 0;
    for (int i = 0; i < count; ++i) {
      const ash_hologram* h = b->holos[i];
      blocks += (h->g.N + kTcRows - 1) / kTcRows;
      fd[i] = TcFieldDesc{h->g, h->amp_img, h->wgs_phase, h->fimg};
      tiles0[i] = t0;
      t0 += h->g.T;
    }
    b->cap_begin = 2 * gmax + 4 * (size_t)count + 4;
    b->cap_split = (2 * gmax + 2 * (size_t)count) * 2 * kTcRows;
    b->cap_fix = gmax + blocks + (size_t)count;
    if (cudaMalloc(&b->d_adj, sizeof(TcAdjParams) * count) || cudaMalloc(&b->d_fwd, sizeof(TcFwdParams) * count) ||
        cudaMalloc(&b->d_hu0, sizeof(long long) * 2 * (count + 1)) || cudaMalloc(&b->d_g0, sizeof(int) * 2 * count) ||
        cudaMalloc(&b->d_begin, sizeof(long long) * b->cap_begin) ||
        cudaMalloc(&b->d_tsplit, sizeof(float2) * b->cap_split) || cudaMalloc(&b->d_lists, sizeof(int4) * b->cap_fix) ||
        cudaMalloc(&b->d_field, sizeof(TcFieldDesc) * count) || cudaMalloc(&b->d_tiles0, sizeof(int) * count)) {
      cudaGetLastError();
      return fail(ASH_ERR_OOM, "batch tensor-core table allocation");
    }
    if ((e = cudaMemcpy(b->d_field, fd.data(), sizeof(TcFieldDesc) * count, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->d_tiles0, tiles0.data(), sizeof(int) * count, cudaMemcpyHostToDevice)))
      return status_cuda(e, "batch tensor-core descriptors");
  }
  return set_grid(b, b->use_tc() ? b->tc_slots : b->slots);
}

// Autotuner cache key: the device's SM count and, per member in order, its
// bucketed shape (log2 of the pixel count and of the spot count, rounded
// up) and its mode count.
std::string tune_key(const ash_batch* b) {
  auto lg = [](long long v) {
    int k = 0;
    while ((1LL << k) < v) ++k;
    return k;
  };
  std::string key = "sm" + std::to_string(b->sms);
  for (const ash_hologram* h : b->all)
    key += "_m" + std::to_string(lg((long long)h->g.nx * h->g.ny)) + "n" + std::to_string(lg(h->g.N)) + "d" +
           std::to_string(h->g.D);
  return key;
}

// The batch's WGS loop for `iters` iterations (standalone members' loops
// and the persistent group's launches) captured and instantiated.
ash_status capture_loop(ash_batch* b, int iters, cudaGraphExec_t* exec, int* kernels) {
  cudaGraph_t graph = nullptr;
  BCUDA(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
  ash_status st = ASH_OK;
  for (ash_hologram* h : b->solo)
    if (st == ASH_OK) st = wgs_body(h, iters, b->capture);
  if (st == ASH_OK && b->count > 0) st = enqueue_batch_body(b, iters, b->capture);
  cudaError_t ce = cudaStreamEndCapture(b->capture, &graph);
  if (st != ASH_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return status_cuda(ce, "batch cudaStreamEndCapture");
  if (kernels) *kernels = graph_kernel_nodes(graph);
  ce = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return status_cuda(ce, "batch cudaGraphInstantiate");
  return ASH_OK;
}

// Autotuner cache: text lines "key solo_terms family grid"; the last line
// with the batch's key wins.
struct TuneChoice {
  long long solo_terms = -1;
  int family = 0;   // the batch's kernel variant: 0 automatic (tensor core where possible), 1 FMA pipe
  int grid = 0;
};

bool cache_lookup(const char* path, const std::string& key, TuneChoice* out) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  std::vector<char> line(1 << 16);
  bool found = false;
  while (fgets(line.data(), (int)line.size(), f)) {
    const std::string l(line.data());
    const size_t sp = l.find(' ');
    if (sp != key.size() || l.compare(0, sp, key) != 0) continue;
    TuneChoice c;
    if (sscanf(l.c_str() + sp, " %lld %d %d", &c.solo_terms, &c.family, &c.grid) == 3 && c.solo_terms >= 0 &&
        (c.family == 0 || c.family == 1) && c.grid >= 0) {
      *out = c;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const TuneChoice& c) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %lld %d %d\n", key.c_str(), c.solo_terms, c.family, c.grid);
  fclose(f);
}

// Apply a tuned choice: grouping, kernel family, persistent grid.
ash_status apply_choice(ash_batch* b, const TuneChoice& c, cudaStream_t s) {
  b->variant = c.family;
  ash_status st = build_group(b, c.solo_terms, s);
  if (st != ASH_OK) return st;
  if (b->count > 0 && c.grid > 0) st = set_grid(b, c.grid);
  return st;
}

__global__ void k_fill_f(float* __restrict__ x, int n, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

}  // namespace

extern "C" {

ash_status ash_batch_create(ash_batch** out, int count, const ash_hologram_desc* descs, void* stream) {
  return ash_batch_create_ex(out, count, descs, kBatchSoloTerms, stream);
}

ash_status ash_batch_create_ex(ash_batch** out, int count, const ash_hologram_desc* descs, long long solo_terms,
                               void* stream) {
  if (!out) return fail(ASH_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || count > 65535 || !descs) return fail(ASH_ERR_INVALID_ARG, "count outside [1, 65535] or NULL descs");
  if (solo_terms < 0) return fail(ASH_ERR_INVALID_ARG, "solo_terms < 0");
  auto is_solo = [&](const ash_hologram_desc& d) { return (long long)d.N * d.nx * d.ny >= solo_terms; };
  for (int i = 0; i < count; ++i)
    if (!is_solo(descs[i]) && (descs[i].D < 1 || descs[i].D > kBatchMaxD))
      return fail(ASH_ERR_UNSUPPORTED, "batched holograms need 1 <= D <= 12 (hologram " + std::to_string(i) + ")");
  if (consume_injected_failure()) return fail(ASH_ERR_INJECTED, "injected failure");
  ash_batch* b = new ash_batch();
  b->members = count;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto bail = [&](ash_status st) {
    destroy_batch(b);
    return st;
  };
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  for (int i = 0; i < count; ++i) {
    const ash_hologram_desc& d = descs[i];
    ash_hologram* h = nullptr;
    ash_status st = ash_hologram_create(&h, d.nx, d.ny, d.amp, d.D, d.noll, d.basis, d.N, d.coeff, stream);
    if (st != ASH_OK) return bail(st);
    b->all.push_back(h);
  }
  cudaError_t e0 = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e0 != cudaSuccess) return bail(status_cuda(e0, "batch capture stream"));
  ash_status st = build_group(b, solo_terms, s);
  if (st != ASH_OK) return bail(st);
  *out = b;
  return ASH_OK;
}

void ash_batch_destroy(ash_batch* b) {
  if (b) destroy_batch(b);
}

ash_status ash_batch_info(const ash_batch* b, int* count, int* grid, int* resident_ctas, long long* units) {
  if (!b) return fail(ASH_ERR_INVALID_ARG, "batch is NULL");
  if (count) *count = b->members;
  if (grid) *grid = b->G;
  if (resident_ctas) *resident_ctas = b->use_tc() ? b->tc_slots : b->slots;
  if (units) *units = b->U;
  return ASH_OK;
}

ash_status ash_batch_set_grid(ash_batch* b, int grid) {
  if (!b || grid < 1) return fail(ASH_ERR_INVALID_ARG, "NULL batch or grid < 1");
  return set_grid(b, grid);
}

ash_status ash_batch_set_variant(ash_batch* b, int variant) {
  if (!b || variant < 0 || variant > 2) return fail(ASH_ERR_INVALID_ARG, "variant must be 0, 1 or 2");
  if (variant == 2 && b->count > 0 && !b->tc_ok)
    return fail(ASH_ERR_UNSUPPORTED, "tensor-core batch needs every hologram with the same K-atom count (D <= 21)");
  for (ash_hologram* h : b->solo)
    if (variant == 2 && !h->tc_ok)
      return fail(ASH_ERR_UNSUPPORTED, "a standalone member has no tensor-core path (D > 21)");
  for (ash_hologram* h : b->solo) {
    const ash_status st = ash_set_kernel_variant(h, variant);
    if (st != ASH_OK) return st;
  }
  b->variant = variant;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
  b->graph_kernels.clear();
  b->G = 0;
  return set_grid(b, b->use_tc() ? b->tc_slots : b->slots);
}

int ash_batch_standalone(const ash_batch* b) { return b ? (int)b->solo.size() : -1; }

int ash_batch_graph_kernels(const ash_batch* b, int iters) {
  if (!b) return -1;
  auto it = b->graph_kernels.find(iters);
  return it == b->graph_kernels.end() ? -1 : it->second;
}

int ash_batch_wgs_launches(const ash_batch* b, int iters) {
  if (!b || iters < 0) return -1;
  int solo = 0;
  for (const ash_hologram* h : b->solo) solo += ash_wgs_launches(h, iters);
  if (b->count == 0) return solo;
  if (b->use_tc()) {
    const int fwd = 1 + (b->n_red > 0 ? 1 : 0), adj = 1 + (b->n_fix > 0 ? 1 : 0);
    return solo + 1 + fwd + iters * (1 + adj + fwd) + 1;   // nearfield images, forward, iterations, metrics
  }
  const int fwd = 2, adj = b->split ? 2 : 1;
  return solo + iters * (fwd + 1 + adj) + fwd + 1;
}

ash_status ash_batch_wgs(ash_batch* b, float* const* phases, float* const* weights, const float* const* targets,
                         int iters, float* metrics_out, void* stream) {
  if (!b || !phases || !weights || !targets) return fail(ASH_ERR_INVALID_ARG, "NULL argument");
  if (iters < 0 || iters > 1000000) return fail(ASH_ERR_INVALID_ARG, "iters outside [0, 1e6]");
  for (int i = 0; i < b->members; ++i)
    if (!phases[i] || !weights[i] || !targets[i]) return fail(ASH_ERR_INVALID_ARG, "NULL per-hologram buffer");
  if (consume_injected_failure()) return fail(ASH_ERR_INJECTED, "injected failure");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < b->members; ++i) {
    const ash_hologram* h = b->all[i];
    const size_t M = (size_t)h->g.nx * h->g.ny, N = (size_t)h->g.N;
    BCUDA(cudaMemcpyAsync(h->wgs_phase, phases[i], M * 4, cudaMemcpyDeviceToDevice, s));
    BCUDA(cudaMemcpyAsync(h->wgs_w, weights[i], N * 4, cudaMemcpyDeviceToDevice, s));
    BCUDA(cudaMemcpyAsync(h->wgs_T, targets[i], N * 4, cudaMemcpyDeviceToDevice, s));
  }
  auto it = b->graphs.find(iters);
  cudaGraphExec_t exec = nullptr;
  if (it != b->graphs.end()) {
    exec = it->second;
  } else {
    int kernels = 0;
    ash_status st = capture_loop(b, iters, &exec, &kernels);
    if (st != ASH_OK) return st;
    b->graphs[iters] = exec;
    b->graph_kernels[iters] = kernels;
  }
  BCUDA(cudaGraphLaunch(exec, s));
  for (int i = 0; i < b->members; ++i) {
    const ash_hologram* h = b->all[i];
    const size_t M = (size_t)h->g.nx * h->g.ny, N = (size_t)h->g.N;
    BCUDA(cudaMemcpyAsync(phases[i], h->wgs_phase, M * 4, cudaMemcpyDeviceToDevice, s));
    BCUDA(cudaMemcpyAsync(weights[i], h->wgs_w, N * 4, cudaMemcpyDeviceToDevice, s));
    if (metrics_out)
      BCUDA(cudaMemcpyAsync(metrics_out + 4 * i, h->wgs_metrics, 16, cudaMemcpyDeviceToDevice, s));
  }
  return ASH_OK;
}

ash_status ash_batch_tune(ash_batch* b, const float* const* phases, const char* cache_path, int* grid_out,
                          void* stream) {
  if (!b || !phases) return fail(ASH_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < b->members; ++i)
    if (!phases[i]) return fail(ASH_ERR_INVALID_ARG, "NULL per-hologram phase");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // a kernel family forced with ash_batch_set_variant is kept; the automatic
  // one is tuned between the tensor-core and the FMA-pipe kernels
  const int forced = b->variant;
  const std::string key = tune_key(b) + (forced ? "_v" + std::to_string(forced) : std::string());
  TuneChoice hit;
  if (cache_lookup(cache_path, key, &hit)) {
    ash_status st = apply_choice(b, hit, s);
    if (st != ASH_OK) return st;
    if (grid_out) *grid_out = b->G;
    return ASH_OK;
  }
  if (consume_injected_failure()) return fail(ASH_ERR_INJECTED, "injected failure");
  // the timed loops run on the caller's phases with unit weights and targets
  for (int i = 0; i < b->members; ++i) {
    ash_hologram* h = b->all[i];
    const int N = h->g.N;
    BCUDA(cudaMemcpyAsync(h->wgs_phase, phases[i], (size_t)h->g.nx * h->g.ny * 4, cudaMemcpyDeviceToDevice, s));
    k_fill_f<<<(N + 255) / 256, 256, 0, s>>>(h->wgs_w, N, 1.0f);
    k_fill_f<<<(N + 255) / 256, 256, 0, s>>>(h->wgs_T, N, 1.0f);
    BCUDA(cudaGetLastError());
  }
  BCUDA(cudaStreamSynchronize(s));
  cudaEvent_t e0, e1;
  BCUDA(cudaEventCreate(&e0));
  BCUDA(cudaEventCreate(&e1));
  // one warm-up call, then `reps` timed calls
  auto elapsed = [&](auto&& fn, int reps, float* ms) -> ash_status {
    ash_status st = fn();
    if (st != ASH_OK) return st;
    BCUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps && st == ASH_OK; ++r) st = fn();
    if (st != ASH_OK) return st;
    BCUDA(cudaEventRecord(e1, s));
    BCUDA(cudaEventSynchronize(e1));
    BCUDA(cudaEventElapsedTime(ms, e0, e1));
    return ASH_OK;
  };
  // candidate groupings: every member standalone, the persistent group for
  // members below 2^20 .. 2^26 terms, every member in the group (those the
  // persistent kernels cannot take stay standalone); distinct ones only
  std::vector<long long> thresholds;
  std::vector<std::vector<bool>> parts;
  for (long long thr : {0LL, 1LL << 20, 1LL << 22, 1LL << 24, 1LL << 26, 1LL << 62}) {
    std::vector<bool> p;
    for (const ash_hologram* h : b->all)
      p.push_back((long long)h->g.N * h->g.nx * h->g.ny >= thr || h->g.D > kBatchMaxD);
    bool seen = false;
    for (const auto& q : parts) seen = seen || q == p;
    if (!seen) {
      parts.push_back(p);
      thresholds.push_back(thr);
    }
  }
  TuneChoice best;
  best.solo_terms = b->solo_terms;
  best.family = forced;
  float best_ms = 1e30f;
  const int kTimedIters = 2;
  ash_status st = ASH_OK;
  const std::vector<int> families = forced ? std::vector<int>{forced} : std::vector<int>{0, 1};
  for (long long thr : thresholds) {
    for (int fam : families) {
      b->variant = fam;
      if ((st = build_group(b, thr, s)) != ASH_OK) break;
      // family 1 on a grouping without a persistent group, or 0 on a group
      // the tensor-core kernels cannot take, repeats the other family's case
      if (families.size() > 1 && fam == 1 && b->count == 0) continue;
      if (families.size() > 1 && fam == 0 && b->count > 0 && !b->tc_ok) continue;
      int grid = 0;
      if (b->count > 0) {
        // launch shape of the persistent group: one forward + adjoint per candidate CTA count
        if (b->use_tc()) BCUDA(tc_field_img_batch(b->d_field, b->d_tiles0, b->count, b->total_tiles, s));
        auto fwd_adj = [&]() -> ash_status {
          if (b->use_tc()) {
            ash_status r = enqueue_tc_forward(b, s);
            return r == ASH_OK ? enqueue_tc_adjoint(b, s) : r;
          }
          ash_status r = enqueue_batch_forward(b, s);
          return r == ASH_OK ? enqueue_batch_adjoint(b, s) : r;
        };
        const int sl = b->use_tc() ? b->tc_slots : b->slots;
        float gbest = 1e30f;
        for (int c : {sl / 2, sl, (3 * sl) / 2, 2 * sl, 3 * sl, 4 * sl}) {
          if (c < 1) continue;
          if ((st = set_grid(b, c)) != ASH_OK) break;
          float ms = 0.0f;
          if ((st = elapsed(fwd_adj, 2, &ms)) != ASH_OK) break;
          if (ms < gbest) {
            gbest = ms;
            grid = b->G;
          }
        }
        if (st == ASH_OK) st = set_grid(b, grid);
        if (st != ASH_OK) break;
      }
      // the whole loop of this choice, as the graph ash_batch_wgs runs
      cudaGraphExec_t exec = nullptr;
      if ((st = capture_loop(b, kTimedIters, &exec, nullptr)) != ASH_OK) break;
      float ms = 0.0f;
      st = elapsed(
          [&]() -> ash_status {
            const cudaError_t ce = cudaGraphLaunch(exec, s);
            return ce == cudaSuccess ? ASH_OK : status_cuda(ce, "tuner graph launch");
          },
          2, &ms);
      cudaGraphExecDestroy(exec);
      if (st != ASH_OK) break;
      if (ms < best_ms) {
        best_ms = ms;
        best.solo_terms = thr;
        best.family = fam;
        best.grid = grid;
      }
    }
    if (st != ASH_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ASH_OK) return st;
  if ((st = apply_choice(b, best, s)) != ASH_OK) return st;
  cache_store(cache_path, key, best);
  if (grid_out) *grid_out = b->G;
  return ASH_OK;
}

}  // extern "C"
