// Set-up and N-length kernels: basis materialisation, layout conversion,
// deterministic column reductions, the weighted-GS spot update and metrics.
// Kernels have internal linkage (static) so the header can serve several
// translation units; the *_body device functions are shared with the
// batched kernels.
#pragma once

#include "common.cuh"
#include "mono.h"

namespace ash {

struct BasisParams {
  Geometry g;
  const MonoTerm* terms;   // all modes' terms, concatenated
  const int* term_off;     // [D + 1] offsets into terms
  int max_order;           // max px or py over all terms
  const float* user_basis; // [D][ny][nx] or null (then terms are used)
  float* dz;               // register image [T][NT][D][P]
  float2* anchors;         // [T][D], or NULL to rebuild dz only
};

__device__ inline double eval_mono(const MonoTerm* __restrict__ terms, int b, int e, const double* xp,
                                   const double* yp) {
  double z = 0.0;
  for (int q = b; q < e; ++q) z = fma(terms[q].coef, xp[terms[q].px] * yp[terms[q].py], z);
  return z;
}

constexpr int kMaxOrder = 24;

// One CTA per tile, NT threads; thread t fills its P pixels x D modes.
static __global__ void k_basis(const BasisParams p) {
  const Geometry& G = p.g;
  const int tile = blockIdx.x, t = threadIdx.x;
  const int P = G.P, NT = G.NT, D = G.D;
  const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
  const int lane = t & 31, w = t >> 5;
  int ia, ja;
  tile_anchor(G, tile, ia, ja);
  double axp[kMaxOrder + 1], ayp[kMaxOrder + 1];
  double xp[kMaxOrder + 1], yp[kMaxOrder + 1];
  if (!p.user_basis) {
    const double xa = grid_x(G, (double)ia), ya = grid_y(G, (double)ja);
    axp[0] = ayp[0] = 1.0;
    for (int o = 1; o <= p.max_order; ++o) {
      axp[o] = axp[o - 1] * xa;
      ayp[o] = ayp[o - 1] * ya;
    }
  }
  const size_t ma = (size_t)ja * G.nx + ia;
  for (int k = 0; k < P; ++k) {
    const int i = tx * kTileX + lane;
    const int j = ty * kTileY + w + (NT / 32) * k;
    const bool valid = (i < G.nx) && (j < G.ny);
    if (!p.user_basis && valid) {
      const double x = grid_x(G, (double)i), y = grid_y(G, (double)j);
      xp[0] = yp[0] = 1.0;
      for (int o = 1; o <= p.max_order; ++o) {
        xp[o] = xp[o - 1] * x;
        yp[o] = yp[o - 1] * y;
      }
    }
    for (int d = 0; d < D; ++d) {
      double v = 0.0;
      if (valid) {
        if (p.user_basis) {
          const size_t plane = (size_t)d * G.nx * G.ny;
          v = (double)p.user_basis[plane + (size_t)j * G.nx + i] - (double)p.user_basis[plane + ma];
        } else {
          const int b = p.term_off[d], e = p.term_off[d + 1];
          v = eval_mono(p.terms, b, e, xp, yp) - eval_mono(p.terms, b, e, axp, ayp);
        }
      }
      p.dz[(((size_t)tile * NT + t) * D + d) * P + k] = (float)v;
    }
  }
  if (t < D && p.anchors) {
    const int d = t;
    double za;
    if (p.user_basis) {
      za = (double)p.user_basis[(size_t)d * G.nx * G.ny + ma];
    } else {
      za = eval_mono(p.terms, p.term_off[d], p.term_off[d + 1], axp, ayp);
    }
    const double turns = za / 6.283185307179586476925286766559;
    const float hi = (float)turns;
    const float lo = (float)(turns - (double)hi);
    p.anchors[(size_t)tile * D + d] = make_float2(hi, lo);
  }
}

// Amplitude into the register-image layout (zero outside the grid).
static __global__ void k_amp_image(Geometry G, const float* __restrict__ amp, float* __restrict__ img) {
  const int tile = blockIdx.x, t = threadIdx.x;
  const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
  const int lane = t & 31, w = t >> 5;
  for (int k = 0; k < G.P; ++k) {
    const int i = tx * kTileX + lane;
    const int j = ty * kTileY + w + (G.NT / 32) * k;
    const bool valid = (i < G.nx) && (j < G.ny);
    img[((size_t)tile * G.NT + t) * G.P + k] = valid ? amp[(size_t)j * G.nx + i] : 0.0f;
  }
}

// Block-wide sum in a fixed order (deterministic). All threads get the result.
template <int NTH>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < NTH / 32; ++q) s += red[q];
  return s;
}

// sum_m A_m^2 in fp64 (one block).
static __global__ void k_sum_sq(const float* __restrict__ a, size_t M, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (size_t m = threadIdx.x; m < M; m += blockDim.x) s += (double)a[m] * (double)a[m];
  s = block_sum<1024>(s, red);
  if (threadIdx.x == 0) *out = s;
}

// out[c] = sum_r in[r][c] (r in fixed order). Block (32, 32): 32 columns,
// 32 row lanes; smem tree over the row lanes.
__device__ __forceinline__ void col_reduce_body(const float* __restrict__ in, int rows, int cols,
                                                float* __restrict__ out, int bx) {
  __shared__ float red[32][33];
  const int c = bx * 32 + threadIdx.x;
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

// Deterministic block-wide fp32 sum (fixed shuffle tree, then a fixed tree
// over the warps); every thread receives the result.
template <int NTH>
__device__ __forceinline__ float block_sum_f(float v, float* red) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float s = lane < NTH / 32 ? red[lane] : 0.0f;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Weighted GS spot update (one block of 1024 threads, fp32):
//   E^ = |E|/||E||, T^ = T/||T||, w <- w T^/max(E^, 1e-30), w <- w/||w||,
//   y = w exp(i arg E) (arg 0 -> 0).
// The norms only fix a global scale of w (removed by the renormalisation,
// and arg g is invariant to it), so fp32 sums are sufficient.
// Weighted GS spot update. Variants (feedback exponent p, phase fixing; p = 1
// and no fixing is the plain rule): w <- w (T^/E^)^p, renormalised; the spot
// phase is arg E, stored as a unit phasor in u_store when given, or, when
// u_fixed is given, the stored phasor instead of arg E.
__device__ __forceinline__ void wgs_update_body(const float2* __restrict__ E, float* __restrict__ w,
                                                const float* __restrict__ T, float2* __restrict__ y, int N,
                                                float feedback = 1.0f, const float2* __restrict__ u_fixed = nullptr,
                                                float2* __restrict__ u_store = nullptr) {
  __shared__ float red[32];
  float se = 0.0f, st = 0.0f;
  for (int n = threadIdx.x; n < N; n += 1024) {
    const float2 e = E[n];
    se = fmaf(e.x, e.x, fmaf(e.y, e.y, se));
    st = fmaf(T[n], T[n], st);
  }
  se = block_sum_f<1024>(se, red);
  st = block_sum_f<1024>(st, red);
  const float ne = sqrtf(se), nt = sqrtf(st);
  float sw = 0.0f;
  for (int n = threadIdx.x; n < N; n += 1024) {
    const float2 e = E[n];
    const float ea = sqrtf(e.x * e.x + e.y * e.y);
    const float eh = fmaxf(ea / ne, 1e-30f);
    const float wn = feedback == 1.0f ? w[n] * (T[n] / nt) / eh : w[n] * powf((T[n] / nt) / eh, feedback);
    w[n] = wn;
    sw = fmaf(wn, wn, sw);
  }
  sw = block_sum_f<1024>(sw, red);
  const float nw = sqrtf(sw);
  for (int n = threadIdx.x; n < N; n += 1024) {
    const float wn = w[n] / nw;
    w[n] = wn;
    float2 u;
    if (u_fixed) {
      u = u_fixed[n];
    } else {
      const float2 e = E[n];
      const float ea = sqrtf(e.x * e.x + e.y * e.y);
      u = ea > 0.0f ? make_float2(e.x / ea, e.y / ea) : make_float2(1.0f, 0.0f);
      if (u_store) u_store[n] = u;
    }
    y[n] = make_float2(wn * u.x, wn * u.y);
  }
}

// Finishes a tile whose spot range (units [u_lo, u_lo + N)) was split
// between CTAs b_lo..b_hi of an adjoint launch: sums their partial fields in
// CTA order and applies the epilogue. slot 0 holds a CTA's first tile.
__device__ __forceinline__ void fixup_tile_body(const HoloView& v, const AdjOut& out, const float2* __restrict__ split,
                                                const Schedule& sched, int tile, long long u_lo, int b_lo, int b_hi) {
  const Geometry& G = v.g;
  const int t = threadIdx.x;
  const int P = G.P, NT = G.NT;
  const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
  const int i = tx * kTileX + (t & 31);
  for (int k = 0; k < P; ++k) {
    float gr = 0.0f, gi = 0.0f;
    for (int b = b_lo; b <= b_hi; ++b) {
      const int slot = (sched.begin(b) >= u_lo) ? 0 : 1;
      const float2 val = split[((size_t)b * 2 + slot) * kTilePix + (size_t)k * NT + t];
      gr += val.x;
      gi += val.y;
    }
    const int j = ty * kTileY + (t >> 5) + (NT / 32) * k;
    if (i >= G.nx || j >= G.ny) continue;
    const float a = (out.epilogue & kEpiGradPhase) ? v.amp_img[((size_t)tile * NT + t) * P + k] : 0.0f;
    adjoint_epilogue(out, (size_t)j * G.nx + i, gr, gi, a);
  }
}

// metrics = {uniformity, efficiency, sum |E|^2, min I^} (one block).
__device__ __forceinline__ void metrics_body(const float2* __restrict__ E, const float* __restrict__ T, int N,
                                             const double* __restrict__ sum_a2, double M,
                                             float* __restrict__ metrics) {
  __shared__ double red[32];
  __shared__ float rmin[32], rmax[32];
  double se = 0.0;
  float lo = 3.0e38f, hi = 0.0f;
  for (int n = threadIdx.x; n < N; n += 1024) {
    const float2 e = E[n];
    const float I = e.x * e.x + e.y * e.y;
    se += (double)I;
    const float ih = I / (T[n] * T[n]);
    lo = fminf(lo, ih);
    hi = fmaxf(hi, ih);
  }
  se = block_sum<1024>(se, red);
  for (int o = 16; o >= 1; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  if (lane == 0) {
    rmin[wq] = lo;
    rmax[wq] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < 32; ++q) {
      lo = fminf(lo, rmin[q]);
      hi = fmaxf(hi, rmax[q]);
    }
    lo = fminf(lo, rmin[0]);
    hi = fmaxf(hi, rmax[0]);
    metrics[0] = (hi + lo) > 0.0f ? 1.0f - (hi - lo) / (hi + lo) : 0.0f;
    metrics[1] = (float)(se / (M * (*sum_a2)));
    metrics[2] = (float)se;
    metrics[3] = lo;
  }
}

// Spot-intensity loss (one block, fp64 sums in a fixed order):
//   I = |E|^2, mu = mean I, r = I / mu - t, L = sum r^2,
//   dL/dRe E + i dL/dIm E = 2 G E, G_k = (2 / mu) (r_k - (1/N) sum_n r_n I_n / mu).
__device__ __forceinline__ void spot_loss_body(const float2* __restrict__ E, const float* __restrict__ t, int N,
                                               float* __restrict__ loss, float2* __restrict__ gE) {
  __shared__ double red[32];
  double sI = 0.0;
  for (int n = threadIdx.x; n < N; n += 1024) {
    const float2 e = E[n];
    sI += (double)e.x * e.x + (double)e.y * e.y;
  }
  sI = block_sum<1024>(sI, red);
  const double mu = sI / N;
  double sL = 0.0, sR = 0.0;
  for (int n = threadIdx.x; n < N; n += 1024) {
    const float2 e = E[n];
    const double I = (double)e.x * e.x + (double)e.y * e.y;
    const double r = (mu > 0.0 ? I / mu : 0.0) - (double)t[n];
    sL += r * r;
    sR += mu > 0.0 ? r * I / mu : 0.0;
  }
  sL = block_sum<1024>(sL, red);
  sR = block_sum<1024>(sR, red);
  if (threadIdx.x == 0 && loss) *loss = (float)sL;
  if (!gE) return;
  const double c = sR / N;
  for (int n = threadIdx.x; n < N; n += 1024) {
    const float2 e = E[n];
    const double I = (double)e.x * e.x + (double)e.y * e.y;
    const double r = (mu > 0.0 ? I / mu : 0.0) - (double)t[n];
    const double G = mu > 0.0 ? (2.0 / mu) * (r - c) : 0.0;
    gE[n] = make_float2((float)(2.0 * G * e.x), (float)(2.0 * G * e.y));
  }
}

// ---------------------------------------------------------------------------
// Single-hologram wrappers.

static __global__ void k_col_reduce(const float* __restrict__ in, int rows, int cols, float* __restrict__ out) {
  col_reduce_body(in, rows, cols, out, blockIdx.x);
}

static __global__ void k_fill_c(float2* __restrict__ x, int n, float2 v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

static __global__ void __launch_bounds__(1024) k_wgs_update(const float2* __restrict__ E, float* __restrict__ w,
                                                            const float* __restrict__ T, float2* __restrict__ y,
                                                            int N, float feedback, const float2* __restrict__ u_fixed,
                                                            float2* __restrict__ u_store) {
  wgs_update_body(E, w, T, y, N, feedback, u_fixed, u_store);
}

static __global__ void __launch_bounds__(1024) k_spot_loss(const float2* __restrict__ E, const float* __restrict__ t,
                                                           int N, float* __restrict__ loss, float2* __restrict__ gE) {
  spot_loss_body(E, t, N, loss, gE);
}

static __global__ void __launch_bounds__(1024) k_metrics(const float2* __restrict__ E, const float* __restrict__ T,
                                                         int N, const double* __restrict__ sum_a2, double M,
                                                         float* __restrict__ metrics) {
  metrics_body(E, T, N, sum_a2, M, metrics);
}

// One CTA of G.NT threads per tile; tiles owned by a single CTA return at once.
static __global__ void k_adjoint_fixup(const AdjParams p) {
  const long long u_lo = (long long)blockIdx.x * p.v.g.N, u_hi = u_lo + p.v.g.N - 1;
  const int b_lo = p.sched.owner(u_lo), b_hi = p.sched.owner(u_hi);
  if (b_lo == b_hi) return;
  fixup_tile_body(p.v, p.out, p.split, p.sched, blockIdx.x, u_lo, b_lo, b_hi);
}

}  // namespace ash
