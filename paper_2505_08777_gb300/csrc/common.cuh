// Shared device helpers, geometry and kernel parameter blocks.
//
// Data layout (HBM):
//   The SLM grid is cut into 32 x 32 pixel tiles. Each tile is processed by
//   one CTA of NT = 1024 / P threads; thread t owns P pixels of the tile:
//   column (t % 32), rows (t / 32) + (NT / 32) * k for k = 0..P-1.
//   The basis is stored relative to one anchor pixel per tile
//   (dZ_dm = Z_d(m) - Z_d(anchor)) in a "register image" layout
//   [tile][t][d][k] (fp32), so that each thread loads its D x P values as
//   contiguous 16-byte vectors and the whole tile is one contiguous block.
//   The anchor values are kept per (tile, mode) as Z_d(anchor)/(2 pi) split
//   into an fp32 hi/lo pair.
//
// Phase split (paper Sec. II kernel K_n(m) = exp(-i sum_d C_nd Z_d(m))):
//   C_n . Z_m = 2 pi * base(n, tile) + C_n . dZ_m
//   base(n, tile) = sum_d C_nd Z_d(anchor)/(2 pi), reduced exactly modulo 1
//   with error-free fp32 products; the local phase C_n . dZ_m stays within
//   a few tens of radians, where sin.approx/cos.approx keep ~1e-5 rad.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ash {

constexpr int kTileX = 32;
constexpr int kTileY = 32;
constexpr int kTilePix = kTileX * kTileY;
constexpr int kMaxModes = 16;

struct Geometry {
  int nx, ny;          // grid (for a band: the band's rows)
  int tiles_x, tiles_y;
  int T;               // number of tiles
  int D;               // modes
  int N;               // spots
  int P;               // pixels per thread
  int NT;              // threads per tile CTA (1024 / P)
  int row0;            // first row of this grid within the full SLM grid (0 unless a band)
  int ny_full;         // rows of the full SLM grid (ny unless a band)
};

// Unit-disk coordinates of the full SLM grid (nx x ny_full): pixel (i, j) of
// this grid sits at x = (i - (nx - 1)/2) / R, y = (row0 + j - (ny_full - 1)/2) / R,
// R = min(nx, ny_full) / 2. A band (a block of whole 32-row tile rows of the
// full grid) therefore has the full grid's basis values and tile anchors.
__host__ __device__ inline double grid_radius(const Geometry& g) {
  return 0.5 * (double)(g.nx < g.ny_full ? g.nx : g.ny_full);
}
__host__ __device__ inline double grid_x(const Geometry& g, double i) { return (i - 0.5 * (double)(g.nx - 1)) / grid_radius(g); }
__host__ __device__ inline double grid_y(const Geometry& g, double j) {
  return ((double)g.row0 + j - 0.5 * (double)(g.ny_full - 1)) / grid_radius(g);
}

// Pixels per thread for a given mode count (register budget of the
// pixel-stationary kernels: P * D basis values live in registers).
#ifndef ASH_P_SMALL_D
#define ASH_P_SMALL_D 8
#endif
__host__ __device__ constexpr int pixels_per_thread(int D) { return D <= 12 ? ASH_P_SMALL_D : 4; }

// Launch bounds of the pixel-stationary kernels: with P = 8 (128 threads)
// ask the register allocator for 3 resident CTAs per SM (<= 170 registers,
// which the D <= 12 kernels meet with at most a few bytes of spill).
#ifndef ASH_MIN_BLOCKS
#define ASH_MIN_BLOCKS 3
#endif
#define ASH_BOUNDS(P) __launch_bounds__(kTilePix / (P), ((P) == 8 ? ASH_MIN_BLOCKS : 1))

// ---------------------------------------------------------------------------
// Packed fp32x2 arithmetic (Blackwell FFMA2): one instruction, two lanes of
// work; used for pixel pairs so the phase contraction and complex MAC take
// half the issue slots.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Round to nearest integer on the FP32 pipe (|x| < 2^22): adding and
// subtracting 1.5 * 2^23 leaves the integer part; __fadd_rn keeps the
// compiler from folding the pair.
__device__ __forceinline__ float rint_fma_pipe(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);
}

// base(n, tile) in turns, reduced to [-1/2, 1/2]:
//   sum_d c[d] * (hi[d] + lo[d]), with hi + lo = Z_d(anchor) / (2 pi).
// c[d]*hi[d] = p + e exactly (fma error term); p - rint(p) is exact; the
// running sum is re-reduced after every mode so it never exceeds ~1 turn.
template <int D>
__device__ __forceinline__ float base_turns(const float* c, const float2* anc) {
  float acc = 0.0f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const float p = __fmul_rn(c[d], anc[d].x);
    const float e = __fmaf_rn(c[d], anc[d].x, -p);
    const float r = __fsub_rn(p, rint_fma_pipe(p));
    const float t = __fmaf_rn(c[d], anc[d].y, e);
    acc = __fadd_rn(acc, __fadd_rn(r, t));
    acc = __fsub_rn(acc, rint_fma_pipe(acc));
  }
  return acc;
}

// exp(i * 2 pi * turns) for |turns| <= 1/2, accurate (sincospif).
__device__ __forceinline__ float2 cis_turns(float turns) {
  float s, c;
  sincospif(2.0f * turns, &s, &c);
  return make_float2(c, s);
}

// ---------------------------------------------------------------------------
// Kernel parameter blocks.

enum FwdSource : int { kSrcPhase = 0, kSrcField = 1 };
// kEpiFimg (tensor-core adjoint only): also write f = A exp(i arg g) in the
// forward's tc layout, so the next WGS forward needs no sincos of its own.
enum AdjEpilogue : int { kEpiField = 1, kEpiPhase = 2, kEpiGradPhase = 4, kEpiFimg = 8 };

// Anchor pixel of a tile: centre of its in-grid part.
__host__ __device__ inline void tile_anchor(const Geometry& g, int tile, int& ia, int& ja) {
  const int tx = tile % g.tiles_x, ty = tile / g.tiles_x;
  const int x0 = tx * kTileX, y0 = ty * kTileY;
  const int x1 = min(x0 + kTileX, g.nx), y1 = min(y0 + kTileY, g.ny);
  ia = (x0 + x1 - 1) / 2;
  ja = (y0 + y1 - 1) / 2;
}

// sin and cos of two local phases on the MUFU pipe (the phases are kept
// small by the tile anchoring, where sin.approx / cos.approx are accurate).
// Polynomial coefficients of sincos2_poly (gen_sincos_poly.py, degree 4 / 4).
__device__ constexpr float kSinPoly[5] = {4.442883015e+00f, -7.308241367e+00f, 3.606288671e+00f, -8.457621932e-01f, 1.092032865e-01f};
__device__ constexpr float kCosPoly[5] = {1.414213538e+00f, -6.978850842e+00f, 5.739460468e+00f, -1.883557916e+00f, 3.106880188e-01f};

__device__ __forceinline__ void sincos2(float2 x, float2& s, float2& c) {
  s.x = __sinf(x.x);
  c.x = __cosf(x.x);
  s.y = __sinf(x.y);
  c.y = __cosf(x.y);
}

// x - 2 pi rint(x / 2 pi) for two arguments (|x| < 2^22): the quotient's
// rint on the FP32 pipe, then the product with 2 pi in two pieces whose high
// part 6.28125 has 8 significant bits, so that k * 6.28125 is exact for
// |k| < 2^16 and each fused step rounds once. The MUFU's sin.approx /
// cos.approx error is about 3.4e-7 for |x| <= pi and grows about
// 1.35e-7 |x| beyond, so reduced arguments keep the transforms' per-term
// error near the fp32 rounding of the phase itself. 5 packed instructions.
__device__ __forceinline__ float2 reduce_2pi2(float2 x) {
  const float2 one = make_float2(1.0f, 1.0f);
  const float2 magic = make_float2(12582912.0f, 12582912.0f), nmagic = make_float2(-12582912.0f, -12582912.0f);
  const float2 t = mul2(x, make_float2(0.159154943091895336f, 0.159154943091895336f));
  const float2 k = fma2(fma2(t, one, magic), one, nmagic);   // rint(t)
  const float2 r = fma2(k, make_float2(-6.28125f, -6.28125f), x);
  return fma2(k, make_float2(-1.9353071795864769e-3f, -1.9353071795864769e-3f), r);
}

// How the transforms feed the MUFU (ASH_MUFU_MODE): 0 the phase as it is;
// 1 the phase reduced to [-pi, pi] first (reduce_2pi2); 2 the phase scaled
// by 1 + kMufuBias. Measured on GB300 against float64 over |x| <= 33 rad:
// sin.approx / cos.approx return the sine and cosine of a phase shrunk by
// 6e-8 .. 9e-8 of itself (mean 7.5e-8, varying with the binade of
// x / 2 pi), with a random part of about a third of that, so scaling the
// argument by 1 + 7.5e-8 (one packed FMA per pair) removes most of the
// systematic error that reduction removes with five.
#ifndef ASH_MUFU_MODE
#define ASH_MUFU_MODE 1
#endif
constexpr float kMufuBias = 7.5e-8f;
__device__ __forceinline__ float2 mufu_arg2(float2 x) {
  if constexpr (ASH_MUFU_MODE == 1) {
    return reduce_2pi2(x);
  } else if constexpr (ASH_MUFU_MODE == 2) {
    return fma2(x, make_float2(kMufuBias, kMufuBias), x);
  } else {
    return x;
  }
}
__device__ __forceinline__ void sincos2_reduced(float2 x, float2& s, float2& c) { sincos2(mufu_arg2(x), s, c); }

// sin and cos of two arguments on the FP32 pipe (packed FFMA2), to share the
// transforms' sincos load between the MUFU and the FP32 pipes. Reduction to
// the half angle: t = x / (2 pi), r = t - rint(t) in [-1/2, 1/2] (rint by
// adding and subtracting 1.5 * 2^23, exact for |t| < 2^22), u = r^2; S(u) ~
// sqrt(2) sin(pi r) / r and C(u) ~ sqrt(2) cos(pi r) are polynomials of
// degree 4 in u, so sin x = 2 sin(pi r) cos(pi r) = (r S) C and
// cos x = 2 cos^2(pi r) - 1 = C^2 - 1. Coefficients: a weighted
// least-squares fit on Chebyshev nodes, written by gen_sincos_poly.py;
// absolute error below 5e-7 on both (that script's float32 bound; the GPU
// test checks the device function against float64).
// sin(2 pi t) and cos(2 pi t) on the FP32 pipe for two phases t in turns:
// r = t - rint(t) is exact, u = r^2, and the polynomials below.
__device__ __forceinline__ void sincos2_poly_turns(float2 t, float2& s, float2& c) {
  const float2 one = make_float2(1.0f, 1.0f), mone = make_float2(-1.0f, -1.0f);
  const float2 magic = make_float2(12582912.0f, 12582912.0f), nmagic = make_float2(-12582912.0f, -12582912.0f);
  const float2 k = fma2(fma2(t, one, magic), one, nmagic);   // rint(t)
  const float2 r = fma2(k, mone, t);
  const float2 u = mul2(r, r);
  float2 S = fma2(u, make_float2(kSinPoly[4], kSinPoly[4]), make_float2(kSinPoly[3], kSinPoly[3]));
  S = fma2(S, u, make_float2(kSinPoly[2], kSinPoly[2]));
  S = fma2(S, u, make_float2(kSinPoly[1], kSinPoly[1]));
  S = fma2(S, u, make_float2(kSinPoly[0], kSinPoly[0]));
  float2 C = fma2(u, make_float2(kCosPoly[4], kCosPoly[4]), make_float2(kCosPoly[3], kCosPoly[3]));
  C = fma2(C, u, make_float2(kCosPoly[2], kCosPoly[2]));
  C = fma2(C, u, make_float2(kCosPoly[1], kCosPoly[1]));
  C = fma2(C, u, make_float2(kCosPoly[0], kCosPoly[0]));
  s = mul2(mul2(r, S), C);
  c = fma2(C, C, mone);
}

__device__ __forceinline__ void sincos2_poly(float2 x, float2& s, float2& c) {
  // t = x / (2 pi); unless ASH_MUFU_MODE is 0 the fp32 constant's rounding
  // (-4e-8 of it) is made up by a second term
  float2 t = mul2(x, make_float2(0.159154943091895336f, 0.159154943091895336f));
  if constexpr (ASH_MUFU_MODE != 0) t = fma2(x, make_float2(6.4206382e-09f, 6.4206382e-09f), t);
  sincos2_poly_turns(t, s, c);
}

// Which pixel pairs of an unrolled loop take the FP32-pipe sincos: NUM of
// every 9, spread evenly. Per pair the MUFU path costs 32 MUFU-pipe cycles
// per warp (4 sin/cos at 16 per clk per SM) and ~10 FP32-pipe cycles (~20
// with the argument reduction), the FP32 path ~40 FP32-pipe cycles; the
// measured best share is lower than the pipe balance (the polynomial's
// dependent chains add latency) and depends on the kernel's own FP32 work:
// ASH_POLY_FWD / _ADJ / _GRAD of 9. Measured on GB300 with the reduced MUFU
// arguments (c2 1024^2 N = 400 / c4 N = 1024 / c3, forward and adjoint us):
// 0/9 277.6, 290.7 / 620.2, 688.1 / 2615, 2845; 2/9 273.4, 292.8 / 609.6,
// 694.3 / 2570, 2844; 3/9 267.3, 298.9 / 601.2, 706.5 / 2544, 2954; 4/9
// 273.4, 307.1 / 621.6, 714.7 / 2634, 3086: 3/9 in the forward, 0/9 in the
// adjoint. The moment pass needs one sine per pixel, not a sine and a
// cosine, and its FP32 pipe also carries the moments: 0/9 (1/9 is 5 %
// slower).
#ifndef ASH_POLY_FWD
#define ASH_POLY_FWD 3
#endif
#ifndef ASH_POLY_ADJ
#define ASH_POLY_ADJ 0
#endif
#ifndef ASH_POLY_GRAD
#define ASH_POLY_GRAD 0
#endif
template <int NUM>
__device__ __forceinline__ void sin2_mixed(int k, float2 x, float2& s) {
  if (NUM > 0 && (k * NUM) % 9 < NUM) {
    float2 c;
    sincos2_poly(x, s, c);   // the cosine's last step is dead code here
  } else {
    const float2 r = mufu_arg2(x);
    s.x = __sinf(r.x);
    s.y = __sinf(r.y);
  }
}

template <int NUM>
__device__ __forceinline__ void sincos2_mixed(int k, float2 x, float2& s, float2& c) {
  if (NUM > 0 && (k * NUM) % 9 < NUM) {
    sincos2_poly(x, s, c);
  } else {
    sincos2_reduced(x, s, c);
  }
}

// The same for phases in turns (the tensor-core transforms: their operand
// rows carry C / 2 pi and their nearfield images phases / 2 pi, so the
// reduction r = t - rint(t) is exact and costs two packed instructions plus
// the subtraction; the MUFU then gets 2 pi r, |2 pi r| <= pi).
__device__ __forceinline__ float2 mufu_arg2_turns(float2 t) {
  const float2 tp = make_float2(6.283185307179586f, 6.283185307179586f);
  if constexpr (ASH_MUFU_MODE == 1) {
    const float2 one = make_float2(1.0f, 1.0f), mone = make_float2(-1.0f, -1.0f);
    const float2 magic = make_float2(12582912.0f, 12582912.0f), nmagic = make_float2(-12582912.0f, -12582912.0f);
    const float2 k = fma2(fma2(t, one, magic), one, nmagic);
    return mul2(fma2(k, mone, t), tp);
  } else if constexpr (ASH_MUFU_MODE == 2) {
    return mufu_arg2(mul2(t, tp));
  } else {
    return mul2(t, tp);
  }
}

// REDUCE = false feeds the MUFU 2 pi t unreduced: its error then grows as
// ~7.5e-8 |2 pi t| (a bias), harmless for a single pass such as the
// gradient's moments (|t| is a tile's local phase, tens of turns at most)
// but not for the transforms a WGS loop repeats.
template <int NUM, bool REDUCE = true>
__device__ __forceinline__ void sin2_turns_mixed(int k, float2 t, float2& s) {
  if (NUM > 0 && (k * NUM) % 9 < NUM) {
    float2 c;
    sincos2_poly_turns(t, s, c);   // the cosine's last step is dead code here
  } else {
    const float2 r = REDUCE ? mufu_arg2_turns(t) : mul2(t, make_float2(6.283185307179586f, 6.283185307179586f));
    s.x = __sinf(r.x);
    s.y = __sinf(r.y);
  }
}

template <int NUM, bool REDUCE = true>
__device__ __forceinline__ void sincos2_turns_mixed(int k, float2 t, float2& s, float2& c) {
  if (NUM > 0 && (k * NUM) % 9 < NUM) {
    sincos2_poly_turns(t, s, c);
  } else {
    sincos2(REDUCE ? mufu_arg2_turns(t) : mul2(t, make_float2(6.283185307179586f, 6.283185307179586f)), s, c);
  }
}

// Balanced static schedule: the T * N (tile, spot) work units, tile-major,
// are cut into G equal contiguous ranges, one per CTA. A tile whose spots
// fall into two or more ranges is finished by the adjoint fix-up pass.
struct Schedule {
  long long W;   // T * N
  int G;         // CTAs
  __host__ __device__ long long begin(int b) const { return ((long long)b * W) / G; }
  // CTA owning work unit u
  __host__ __device__ int owner(long long u) const {
    int b = (int)((u * (long long)G) / W);
    while (b + 1 < G && begin(b + 1) <= u) ++b;
    while (b > 0 && begin(b) > u) --b;
    return b;
  }
};

// Everything a tile computation needs to know about one hologram.
struct HoloView {
  Geometry g;
  const float* dz;        // register-image basis [T][NT][D][P]
  const float* amp_img;   // register-image amplitude [T][NT][P]
  const float2* anchors;  // [T][D] (hi, lo) of Z(anchor)/(2 pi)
  const float* coeff;     // [N][D]
};

struct FwdParams {
  HoloView v;
  Schedule sched;
  const float* phase;     // user layout [ny][nx] (kSrcPhase)
  const float2* field;    // user layout [ny][nx] complex (kSrcField)
  int source;
  float* partial;         // [T * NW][2N]: row (tile, warp), each entry written once
};

// Where the adjoint's per-pixel results go.
struct AdjOut {
  float2* g_out;          // user layout complex or null
  float* phase_out;       // user layout or null
  const float* phase_in;  // for kEpiGradPhase: current phase (user layout)
  float* dphase;          // for kEpiGradPhase
  int epilogue;
};

struct AdjParams {
  HoloView v;
  Schedule sched;
  const float2* y;        // [N] complex
  AdjOut out;
  float2* split;          // [G][2][kTilePix]: partial g of tiles split between CTAs
};

// Per-pixel adjoint epilogue (m = flat pixel index, a = amplitude there).
__device__ __forceinline__ void adjoint_epilogue(const AdjOut& o, size_t m, float gr, float gi, float a) {
  if (o.epilogue & kEpiField) o.g_out[m] = make_float2(gr, gi);
  if (o.epilogue & kEpiPhase) o.phase_out[m] = (gr == 0.0f && gi == 0.0f) ? 0.0f : atan2f(gi, gr);
  if (o.epilogue & kEpiGradPhase) {
    float s, c;
    sincosf(__ldg(o.phase_in + m), &s, &c);
    o.dphase[m] = (a * c) * gi - (a * s) * gr;   // -Im(f conj(h)), f = a exp(i phase)
  }
}

struct GradCParams {
  HoloView v;
  const float* phase;     // user layout
  const float2* gradE;    // [N]
  float* partial;         // [gridDim.x][N][D]
};

// Coefficient-gradient kernel shape: threads per CTA, spots per thread.
constexpr int kGradThreads = 128;
constexpr int kGradSpots = 4;

// Device-side error word bits.
constexpr unsigned kErrBadArg = 1u;

}  // namespace ash
