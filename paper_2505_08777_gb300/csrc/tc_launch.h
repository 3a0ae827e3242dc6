// Tensor-core transform path: shapes, operand-image layouts, schedules,
// parameter blocks and launchers (kernels in tc_kernels.cuh, tc.cu).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "mono.h"

namespace ash {

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;                           // M of one MMA
constexpr int kTcChunk = 64;                           // N of one MMA
constexpr int kTcChunksPerTile = kTilePix / kTcChunk;  // 16 chunks of 64 pixels
constexpr int kTcGroupsPerTile = kTilePix / kTcRows;   // 8 groups of 128 pixels
constexpr unsigned kTcWaitPolls = 1u << 24;
constexpr unsigned kErrTimeout = 2u;
constexpr unsigned kErrClaim = 4u;      // a forward CTA found no range to claim
constexpr int kTcMaxModes = 21;                        // 3 D <= 64

// K layout of the operand rows. Regular: the pixel row [hi | lo | hi] and the
// spot row [hi | hi | lo] of the D basis values / coefficients (3 D slots).
// Tilt-exact (when the basis holds the x and y tilts, Noll 2 and 3): across
// a tile the tilts change by exactly (i - i_anchor) / R and (j - j_anchor) /
// R, so the pixel row carries the integer offsets di, dj (exact in tf32) and
// the spot row c_x / R and c_y / R split into tf32 pieces, TP slots per tilt:
//   pixel [hi | lo | hi (other D - 2 modes) | di .. di  dj .. dj ]
//   spot  [hi | hi | lo (other D - 2 modes) | x pieces  y pieces ]
// Every product di * piece is exact, so the tilts' part of the local phase
// carries only the error of splitting c / R: 2^-22 of it with two pieces,
// about 2^-33 with three. Three pieces are used when they fit one K-atom
// (D <= 10), two when only those fit (D = 11, which then needs one K-atom
// instead of two); the regular layout keeps bases without both tilts.
struct TcLayout {
  int D;
  int NA;        // K-atoms of 32 tf32 per row
  int tx, ty;    // positions of the x / y tilt among the D modes (tilt-exact), else -1
  float R;       // min(nx, ny_full) / 2 (grid_radius)
  int tpx, tpy;  // tf32 pieces of the x / y tilt's c / R (tilt-exact: 2 or 3)
};
__host__ __device__ constexpr int tc_na(int D) { return 3 * D <= 32 ? 1 : 2; }
inline TcLayout tc_layout(int D, const int* noll, const Geometry& g) {
  TcLayout L{D, tc_na(D), -1, -1, (float)grid_radius(g), 0, 0};
  if (noll && D >= 2) {
    int tx = -1, ty = -1;
    for (int d = 0; d < D; ++d) {
      if (noll[d] == 2) tx = d;
      if (noll[d] == 3) ty = d;
    }
    // as many pieces as one K-atom holds: three each, else three for x
    // and two for y, else two each
    const int room = 32 - 3 * (D - 2);
    if (tx >= 0 && ty >= 0 && room >= 4) {
      const int tpx = room >= 5 ? 3 : 2, tpy = room >= 6 ? 3 : 2;
      L = TcLayout{D, 1, tx, ty, L.R, tpx, tpy};
    }
  }
  return L;
}
// Slot `col` of a row: kind 0..2 = segment of mode `mode`, 3 = x tilt
// (piece `mode`, 0 = hi), 4 = y tilt, -1 = padding.
__host__ __device__ inline void tc_slot(const TcLayout& L, int col, int& kind, int& mode) {
  kind = -1;
  mode = 0;
  if (L.tx < 0) {
    if (col < 3 * L.D) {
      kind = col / L.D;
      mode = col % L.D;
    }
    return;
  }
  const int Dp = L.D - 2;
  if (col < 3 * Dp) {
    kind = col / Dp;
    int k = col % Dp;   // k-th mode that is not a tilt
    for (int d = 0; d < L.D; ++d) {
      if (d == L.tx || d == L.ty) continue;
      if (k-- == 0) {
        mode = d;
        break;
      }
    }
  } else if (col < 3 * Dp + L.tpx + L.tpy) {
    const int c = col - 3 * Dp;
    kind = c < L.tpx ? 3 : 4;
    mode = c < L.tpx ? c : c - L.tpx;
  }
}

// Operand images in HBM (floats), each [chunks][NA][64 rows][32] with the
// 128-byte swizzle of tc_common.cuh:
//  zs  : pixel rows, chunk qc = 16 tile + 2 h + half (see tc_pixel);
//  czs : spot rows, chunk j = spots 64 j .. 64 j + 63 (an even number of
//        chunks, rows >= N zero, so a 128-spot block is two chunks), then
//        two chunks holding the last block's spots replicated (tc_fwd_rep);
//  fimg: the nearfield f_m of each pixel chunk as 32 float4 (A, A', phi, phi')
//        of pixel pairs (2p, 2p + 1), phases in turns (phi = arg f / 2 pi).
inline size_t tc_zs_floats(const Geometry& g, int NA) { return (size_t)g.T * kTcChunksPerTile * NA * 2048; }
inline int tc_spot_chunks(int N) { return 2 * ((N + kTcRows - 1) / kTcRows); }
inline size_t tc_czs_floats(int N, int NA) { return (size_t)(tc_spot_chunks(N) + 2) * NA * 2048; }
// The forward's last spot block holds v = N - 128 (nb - 1) spots. With
// v <= 32 (64) its rows are replicated 4 (2) times and each replica's warps
// take a quarter (half) of every pixel chunk, so that the block's work is
// spread over all four warps (and SM sub-partitions) instead of one.
inline int tc_fwd_rep(int N) {
  const int v = N - kTcRows * ((N + kTcRows - 1) / kTcRows - 1);
  return v <= 32 ? 4 : v <= 64 ? 2 : 1;
}
inline size_t tc_fimg_float4s(const Geometry& g) { return (size_t)g.T * kTilePix / 2; }

// Pixel of row r of chunk qc (tile, group h, half): column r % 32, row
// 4 h + 2 half + r / 32 of the tile; `img` is its index in the register-image
// arrays of the FMA kernels (thread t, slot k, P pixels a thread).
struct TcPixel {
  int i, j, tile, img;
};
__host__ __device__ inline TcPixel tc_pixel(const Geometry& G, long long qc, int r) {
  TcPixel px;
  px.tile = (int)(qc / kTcChunksPerTile);
  const int w = (int)(qc % kTcChunksPerTile);
  const int h = w >> 1, half = w & 1;
  const int col = r & 31, row = 4 * h + 2 * half + (r >> 5);
  px.i = (px.tile % G.tiles_x) * kTileX + col;
  px.j = (px.tile / G.tiles_x) * kTileY + row;
  const int rows_per_k = G.NT / 32;
  const int t = (row % rows_per_k) * 32 + col, k = row / rows_per_k;
  px.img = (px.tile * G.NT + t) * G.P + k;
  return px;
}

// Forward schedule: units (spot block b, pixel chunk q), u = b * nq + q, in
// ranges per CTA tabulated on the host (balanced_begins in api.cu). A chunk
// of a partial last block costs as much time as a full one: its time is set
// by the MMA pipeline and its busiest warp, and the warps share their SM
// sub-partitions with the other resident CTAs.
struct TcFwdSched {
  int nb, nq, G;
  __host__ __device__ long long units() const { return (long long)nb * nq; }
  __host__ __device__ long long begin(int g) const { return (long long)g * units() / G; }
  // the CTA whose (non-empty) range contains u
  __host__ __device__ int owner(long long u) const {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (begin(mid) <= u) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
};

// CTA whose (non-empty) range [begin[g], begin[g + 1]) contains unit u.
__host__ __device__ inline int tc_owner(const long long* begin, int G, long long u) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (begin[mid] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Batched launches: the units of `count` holograms concatenated (hologram h
// owns [hu0[h], hu0[h + 1])), cut into G equal CTA ranges; CTA g is local
// CTA g - g0[h] of every hologram it meets.
struct TcBatchSched {
  const long long* hu0;   // [count + 1]
  const int* g0;          // [count]
  int count;
  long long U;
  int G;
  __host__ __device__ long long begin(int g) const { return (long long)g * U / G; }
  __host__ __device__ int holo_of(long long u) const {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (hu0[mid] <= u) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
};

struct TcAdjParams {
  Geometry g;
  const float* zs;
  const float* czs;
  const float2* rot;      // [T][N] exp(+i 2 pi base(n, tile))
  const float2* y;        // [N]
  const float* amp_img;   // register-image amplitude
  AdjOut out;
  float4* fimg;           // written for kEpiFimg
  const long long* begin; // [G + 1] CTA range starts over the units (group, spot chunk of 64),
                          // W = T * 8 * ceil(N / 64) of them
  int G;
  float2* split;          // [G][2][128] partial sums of groups split between CTAs
  const int4* split_groups;  // (group, first CTA, last CTA, -) of the groups whose spots span two or more CTA ranges
  unsigned* err;
};

struct TcFwdParams {
  Geometry g;
  const float* zs;
  const float* czs;
  const float2* rot;
  const float4* fimg;
  TcFwdSched sched;
  int rep;                // tc_fwd_rep(N)
  const long long* begin; // [G + 1] sched.begin(g), tabulated on the host
  float2* E;              // [N]
  float2* part;           // [G][2][128] partial sums of spot blocks split between CTAs
  const int2* spans;      // [nb] first and last CTA meeting each spot block (host-tabulated)
  unsigned* err;
  // SM-aware range claiming (null: CTA g runs range g). Ranges [0, n_full)
  // cover the full spot blocks, [n_full, G) the replicated last block, one
  // per SM: each SM's fourth CTA takes a range of the latter (see
  // tc_claim_range). claim: [0] next full range, [1] next replicated range,
  // [2] CTAs done, [3 + smid] CTAs started on that SM; the last CTA of a
  // launch zeroes it for the next.
  int* claim;
  int n_full;
};
constexpr int kTcClaimSms = 1024;                 // bound on %smid values
constexpr int kTcClaimInts = 3 + kTcClaimSms;

// Coefficient-gradient moments on the tensor cores (one K-atom, D <= 12,
// polynomial basis of total degree ORD <= 4): spot-stationary like the
// forward. tpoly holds, per tile, the basis as polynomials in the pixel's
// column and row offsets: [pairs (k, l), k + l <= ORD][DP modes] floats,
// DP = D rounded up to 4.
constexpr int kTcGradMaxModes = 12, kTcGradMaxOrd = 4;
__host__ __device__ constexpr int tc_grad_dp(int D) { return (D + 3) & ~3; }
__host__ __device__ constexpr int tc_grad_pairs(int ord) { return (ord + 1) * (ord + 2) / 2; }
inline size_t tc_tpoly_floats(const Geometry& g, int ord) {
  return (size_t)g.T * tc_grad_pairs(ord) * tc_grad_dp(g.D);
}
struct TcGradParams {
  Geometry g;
  const float* zs;
  const float* czs;
  const float2* rot;
  const float4* fimg;
  const float* tpoly;
  const float2* gE;       // [N] dL/dE
  TcFwdSched sched;       // units (spot block, pixel chunk), as the forward
  const long long* begin; // [G + 1]
  const int2* spans;      // [nb] first and last CTA meeting each spot block (host-tabulated)
  int ord;                // total degree of the basis polynomials (1..4)
  float* dC;              // [N][D] output
  float* part;            // [G][2][128][DP] partial sums of spot blocks split between CTAs
  unsigned* err;
};
cudaError_t tc_grad_prepare(int ord, int D, int* ctas_per_sm);
cudaError_t tc_build_tile_poly(const Geometry& g, const MonoTerm* terms, const int* term_off, int ord, float* tpoly,
                               cudaStream_t s);
cudaError_t tc_launch_gradc(const TcGradParams& p, bool split, cudaStream_t s);   // kernel (+ reduction of split blocks)
// Resident CTAs per SM from registers, shared memory and TMEM columns.
cudaError_t tc_ctas_per_sm(const void* fn, size_t smem, int tmem_cols, int* out);

// Kernel set-up for operand rows of NA K-atoms: shared-memory limits, and
// resident CTAs per SM from registers, shared memory and TMEM columns.
cudaError_t tc_prepare(int NA, int* adj_ctas_per_sm, int* fwd_ctas_per_sm);
cudaError_t tc_launch_adjoint(int NA, const TcAdjParams& p, int grid, cudaStream_t s);
cudaError_t tc_launch_adjoint_fixup(const TcAdjParams& p, int n_split_groups, cudaStream_t s);
cudaError_t tc_launch_forward(int NA, const TcFwdParams& p, int grid, cudaStream_t s);
cudaError_t tc_launch_forward_reduce(const TcFwdParams& p, cudaStream_t s);
// Batched launches over `count` holograms of the same K-atom count NA;
// device arrays of their parameter blocks, the batch schedule, and the
// fix-up / reduction work lists (hologram, group) and (hologram, spot block).
cudaError_t tc_launch_adjoint_batch(int NA, const TcAdjParams* ps, const TcBatchSched& bs, cudaStream_t s);
cudaError_t tc_launch_adjoint_fixup_batch(const TcAdjParams* ps, const int4* list, int n, cudaStream_t s);
cudaError_t tc_launch_forward_batch(int NA, const TcFwdParams* ps, const TcBatchSched& bs, cudaStream_t s);
cudaError_t tc_launch_forward_reduce_batch(const TcFwdParams* ps, const int4* list, int n, cudaStream_t s);
// Nearfield images of a batch from each hologram's phase (the `phase` of
// its TcFwdParams-sized descriptor below); tiles0[h] = first global tile.
struct TcFieldDesc {
  Geometry g;
  const float* amp_img;
  const float* phase;
  float4* fimg;
};
// Resident CTAs per SM of the batched adjoint and forward kernels.
cudaError_t tc_batch_ctas_per_sm(int NA, int* adj, int* fwd);
cudaError_t tc_field_img_batch(const TcFieldDesc* ds, const int* tiles0, int count, int total_tiles, cudaStream_t s);
cudaError_t tc_build_zs(const Geometry& g, const TcLayout& L, const float* dz, float* zs, cudaStream_t s);
cudaError_t tc_build_coeff(const Geometry& g, const TcLayout& L, const float* coeff, const float2* anchors, float* czs,
                           float2* rot, cudaStream_t s);
cudaError_t tc_field_img(const Geometry& g, const float* amp_img, const float* phase, const float2* field,
                         float4* fimg, cudaStream_t s);

}  // namespace ash
