// Fused spot-kernel transforms: forward E = K f, adjoint g = K^H y, and the
// coefficient-gradient moments. Never forms K: each term's phase
// C_n . dZ_m, its sincos and the complex multiply-accumulate happen in
// registers.
//
// Forward / adjoint are pixel-stationary: a CTA owns one 32x32 tile, each
// thread keeps the basis values of its P pixels in registers, and the CTA
// streams the spots through shared memory in chunks. Per term:
//   D packed FMAs (two pixels per instruction) for the local phase,
//   2 MUFU ops (sin.approx, cos.approx),
//   2 packed FMAs for the complex multiply-accumulate.
// The forward reduces each spot's per-thread partial sums across the warp
// with a transpose reduction (32 values -> one per lane in 5 shuffle stages)
// and rotates the warp sum by exp(-i 2 pi base(n, tile)).
#pragma once

#include "common.cuh"

namespace ash {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSpotChunk = 256;   // spots staged per shared-memory chunk
constexpr int kBatch = 16;        // spots per warp transpose reduction

__host__ __device__ constexpr int cpair_stride(int D) { return ((2 * D) + 3) & ~3; }

// Shared memory bytes of the pixel-stationary kernels.
__host__ __device__ constexpr size_t fwd_smem_bytes(int D) {
  return (size_t)kSpotChunk * cpair_stride(D) * 4 + (size_t)kSpotChunk * 8;
}
__host__ __device__ constexpr size_t adj_smem_bytes(int D) {
  return (size_t)kSpotChunk * cpair_stride(D) * 4 + (size_t)kSpotChunk * 32;
}

// Lane l returns the sum over the warp of a[l].
__device__ __forceinline__ float warp_transpose_reduce32(float (&a)[32], int lane) {
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? a[i] : a[i + half];
      const float keep = up ? a[i + half] : a[i];
      a[i] = keep + __shfl_xor_sync(kFull, send, half);
    }
  }
  return a[0];
}

template <int D, int P>
__device__ __forceinline__ void load_dz(const float* __restrict__ dz_img, int tile, int t,
                                        float2 (&dz)[P / 2][D]) {
  constexpr int NT = kTilePix / P;
  const float4* src = reinterpret_cast<const float4*>(dz_img + ((size_t)tile * NT + t) * D * P);
#pragma unroll
  for (int d = 0; d < D; ++d) {
#pragma unroll
    for (int q = 0; q < P / 4; ++q) {
      const float4 v = __ldg(src + d * (P / 4) + q);
      dz[2 * q][d] = make_float2(v.x, v.y);
      dz[2 * q + 1][d] = make_float2(v.z, v.w);
    }
  }
}

// Stage one spot: duplicated coefficient pairs into sC row, returns base turns.
template <int D>
__device__ __forceinline__ float stage_spot(const float* __restrict__ coeff, const float2* __restrict__ anc,
                                            int n, float* __restrict__ sCrow) {
  float c[D];
  float2 a[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    c[d] = __ldg(coeff + (size_t)n * D + d);
    a[d] = __ldg(anc + d);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    sCrow[2 * d] = c[d];
    sCrow[2 * d + 1] = c[d];
  }
  return base_turns<D>(c, a);
}

template <int D>
__device__ __forceinline__ void load_cpairs(const float* __restrict__ sCrow, float2 (&cc)[D]) {
  const float4* q4 = reinterpret_cast<const float4*>(sCrow);
#pragma unroll
  for (int q = 0; q < D / 2; ++q) {
    const float4 v = q4[q];
    cc[2 * q] = make_float2(v.x, v.y);
    cc[2 * q + 1] = make_float2(v.z, v.w);
  }
  if (D & 1) {
    const float2 v = reinterpret_cast<const float2*>(sCrow)[D - 1];
    cc[D - 1] = v;
  }
}

// Local phase of two pixels (one packed lane each) for one spot.
template <int D>
__device__ __forceinline__ float2 local_phase(const float2 (&cc)[D], const float2 (&z)[D]) {
#if defined(ASH_SPLIT_CHAIN)
  if (D >= 6) {
    // two independent halves shorten the dependent FMA chain
    constexpr int H = D / 2;
    float2 xa = mul2(cc[0], z[0]);
    float2 xb = mul2(cc[H], z[H]);
#pragma unroll
    for (int d = 1; d < H; ++d) xa = fma2(cc[d], z[d], xa);
#pragma unroll
    for (int d = H + 1; d < D; ++d) xb = fma2(cc[d], z[d], xb);
    return make_float2(xa.x + xb.x, xa.y + xb.y);
  }
#endif
  float2 x = mul2(cc[0], z[0]);
#pragma unroll
  for (int d = 1; d < D; ++d) x = fma2(cc[d], z[d], x);
  return x;
}

// ---------------------------------------------------------------------------
// Nearfield pairs f = A exp(i phase) (or a caller field) of a thread's P pixels.
template <int P>
__device__ __forceinline__ void load_field(const HoloView& hv, int source, const float* __restrict__ phase,
                                           const float2* __restrict__ field, int tile, int t,
                                           float2 (&fr2)[P / 2], float2 (&fi2)[P / 2], float2 (&nfr2)[P / 2]) {
  constexpr int NT = kTilePix / P;
  constexpr int RS = NT / 32;
  const Geometry& G = hv.g;
  const int lane = t & 31, w = t >> 5;
  const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
  const int i = tx * kTileX + lane;
  const float4* asrc = reinterpret_cast<const float4*>(hv.amp_img + ((size_t)tile * NT + t) * P);
  float a[P], fr[P], fi[P];
#pragma unroll
  for (int q = 0; q < P / 4; ++q) {
    const float4 v = __ldg(asrc + q);
    a[4 * q] = v.x; a[4 * q + 1] = v.y; a[4 * q + 2] = v.z; a[4 * q + 3] = v.w;
  }
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const int j = ty * kTileY + w + RS * k;
    const bool valid = (i < G.nx) && (j < G.ny);
    const size_t m = (size_t)j * G.nx + i;
    if (source == kSrcPhase) {
      const float ph = valid ? __ldg(phase + m) : 0.0f;
      float sn, cs;
      sincosf(ph, &sn, &cs);
      fr[k] = a[k] * cs;
      fi[k] = a[k] * sn;
    } else {
      const float2 f = valid ? __ldg(field + m) : make_float2(0.0f, 0.0f);
      fr[k] = f.x;
      fi[k] = f.y;
    }
  }
#pragma unroll
  for (int q = 0; q < P / 2; ++q) {
    fr2[q] = make_float2(fr[2 * q], fr[2 * q + 1]);
    fi2[q] = make_float2(fi[2 * q], fi[2 * q + 1]);
    nfr2[q] = make_float2(-fr[2 * q], -fr[2 * q + 1]);
  }
}

// Forward over spots [sb, se) of one tile: ptile[w][2n..2n+1] = sum over
// warp w's pixels of f_m exp(-i C_n . Z_m). Called uniformly by the CTA.
template <int D, int P>
__device__ __forceinline__ void forward_tile(const HoloView& hv, int source, const float* __restrict__ phase,
                                             const float2* __restrict__ field, int tile, int sb, int se,
                                             float* __restrict__ ptile, float* sC, float2* sRot) {
  constexpr int NT = kTilePix / P;
  constexpr int CPS = cpair_stride(D);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int N = hv.g.N;
  float2 dz[P / 2][D];
  load_dz<D, P>(hv.dz, tile, t, dz);
  float2 fr2[P / 2], fi2[P / 2], nfr2[P / 2];
  load_field<P>(hv, source, phase, field, tile, t, fr2, fi2, nfr2);
  float* prow = ptile + (size_t)w * 2 * N;
  const float2* anc = hv.anchors + (size_t)tile * D;

  for (int n0 = sb; n0 < se; n0 += kSpotChunk) {
    const int nc = min(kSpotChunk, se - n0);
    __syncthreads();
    for (int s = t; s < nc; s += NT) {
      const float bt = stage_spot<D>(hv.coeff, anc, n0 + s, sC + s * CPS);
      sRot[s] = cis_turns(-bt);
    }
    __syncthreads();

    for (int b0 = 0; b0 < nc; b0 += kBatch) {
      float acc[32];
#pragma unroll
      for (int s = 0; s < kBatch; ++s) {
        float re = 0.0f, im = 0.0f;
        if (b0 + s < nc) {
          float2 cc[D];
          load_cpairs<D>(sC + (b0 + s) * CPS, cc);
          float2 re2 = make_float2(0.0f, 0.0f), im2 = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int q = 0; q < P / 2; ++q) {
            const float2 x = local_phase<D>(cc, dz[q]);
            float2 sn, cs;
            sincos2_reduced(x, sn, cs);
            re2 = fma2(fr2[q], cs, re2);
            re2 = fma2(fi2[q], sn, re2);
            im2 = fma2(fi2[q], cs, im2);
            im2 = fma2(nfr2[q], sn, im2);
          }
          re = re2.x + re2.y;
          im = im2.x + im2.y;
        }
        acc[2 * s] = re;
        acc[2 * s + 1] = im;
      }
      const float v = warp_transpose_reduce32(acc, lane);
      const float other = __shfl_xor_sync(kFull, v, 1);
      const int s = lane >> 1;
      const bool is_im = (lane & 1) != 0;
      if (b0 + s < nc) {
        const float re = is_im ? other : v;
        const float im = is_im ? v : other;
        const float2 r = sRot[b0 + s];
        prow[2 * (n0 + b0) + lane] = is_im ? fmaf(im, r.x, re * r.y) : fmaf(re, r.x, -im * r.y);
      }
    }
  }
}

// Adjoint over spots [sb, se) of one tile into per-thread accumulators.
template <int D, int P>
__device__ __forceinline__ void adjoint_tile(const HoloView& hv, const float2* __restrict__ y, int tile, int sb,
                                             int se, float2 (&re2)[P / 2], float2 (&im2)[P / 2], float* sC,
                                             float4* sY) {
  constexpr int NT = kTilePix / P;
  constexpr int CPS = cpair_stride(D);
  const int t = threadIdx.x;
  float2 dz[P / 2][D];
  load_dz<D, P>(hv.dz, tile, t, dz);
#pragma unroll
  for (int q = 0; q < P / 2; ++q) {
    re2[q] = make_float2(0.0f, 0.0f);
    im2[q] = make_float2(0.0f, 0.0f);
  }
  const float2* anc = hv.anchors + (size_t)tile * D;
  for (int n0 = sb; n0 < se; n0 += kSpotChunk) {
    const int nc = min(kSpotChunk, se - n0);
    __syncthreads();
    for (int s = t; s < nc; s += NT) {
      const float bt = stage_spot<D>(hv.coeff, anc, n0 + s, sC + s * CPS);
      const float2 r = cis_turns(bt);
      const float2 yv = __ldg(y + n0 + s);
      const float yr = yv.x * r.x - yv.y * r.y;
      const float yi = yv.x * r.y + yv.y * r.x;
      sY[2 * s] = make_float4(yr, yr, yi, yi);
      sY[2 * s + 1] = make_float4(-yi, -yi, 0.0f, 0.0f);
    }
    __syncthreads();

#pragma unroll 2
    for (int s = 0; s < nc; ++s) {
      float2 cc[D];
      load_cpairs<D>(sC + s * CPS, cc);
      const float4 ya = sY[2 * s];
      const float4 yb = sY[2 * s + 1];
      const float2 yr2 = make_float2(ya.x, ya.y);
      const float2 yi2 = make_float2(ya.z, ya.w);
      const float2 nyi2 = make_float2(yb.x, yb.y);
#pragma unroll
      for (int q = 0; q < P / 2; ++q) {
        const float2 x = local_phase<D>(cc, dz[q]);
        float2 sn, cs;
        sincos2_reduced(x, sn, cs);
        re2[q] = fma2(yr2, cs, re2[q]);
        re2[q] = fma2(nyi2, sn, re2[q]);
        im2[q] = fma2(yi2, cs, im2[q]);
        im2[q] = fma2(yr2, sn, im2[q]);
      }
    }
  }
}

// After adjoint_tile: epilogue for a tile whose whole spot range this CTA
// owns, else the partial field into the CTA's split slot.
template <int P>
__device__ __forceinline__ void adjoint_finish(const HoloView& hv, const AdjOut& out, int tile, bool full,
                                               float2* __restrict__ slot, const float2 (&re2)[P / 2],
                                               const float2 (&im2)[P / 2]) {
  constexpr int NT = kTilePix / P;
  constexpr int RS = NT / 32;
  const Geometry& G = hv.g;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (full) {
    const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
    const int i = tx * kTileX + lane;
    const float* aimg = hv.amp_img + ((size_t)tile * NT + t) * P;
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int j = ty * kTileY + w + RS * k;
      if (i >= G.nx || j >= G.ny) continue;
      const float gr = (k & 1) ? re2[k >> 1].y : re2[k >> 1].x;
      const float gi = (k & 1) ? im2[k >> 1].y : im2[k >> 1].x;
      const float a = (out.epilogue & kEpiGradPhase) ? __ldg(aimg + k) : 0.0f;
      adjoint_epilogue(out, (size_t)j * G.nx + i, gr, gi, a);
    }
  } else {
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const float gr = (k & 1) ? re2[k >> 1].y : re2[k >> 1].x;
      const float gi = (k & 1) ? im2[k >> 1].y : im2[k >> 1].x;
      slot[k * NT + t] = make_float2(gr, gi);
    }
  }
}

// ---------------------------------------------------------------------------
// Forward: partial[(tile, warp)][2n..2n+1] over this CTA's (tile, spot) range;
// every entry is written exactly once per launch.
template <int D, int P>
__global__ void ASH_BOUNDS(P) k_forward(const FwdParams p) {
  constexpr int NW = kTilePix / P / 32;
  constexpr int CPS = cpair_stride(D);
  extern __shared__ float4 smem4[];
  float* sC = reinterpret_cast<float*>(smem4);
  float2* sRot = reinterpret_cast<float2*>(sC + kSpotChunk * CPS);
  const int N = p.v.g.N;
  const long long u0 = p.sched.begin(blockIdx.x), u1 = p.sched.begin(blockIdx.x + 1);
  const int tf = (int)(u0 / N), tl = (int)((u1 - 1) / N);
  for (int tile = tf; tile <= tl; ++tile) {
    const int sb = (tile == tf) ? (int)(u0 - (long long)tile * N) : 0;
    const int se = (tile == tl) ? (int)(u1 - (long long)tile * N) : N;
    forward_tile<D, P>(p.v, p.source, p.phase, p.field, tile, sb, se, p.partial + (size_t)tile * NW * 2 * N, sC,
                       sRot);
  }
}

// Adjoint over this CTA's (tile, spot) range. Tiles whose full spot range is
// owned by the CTA get the epilogue here; tiles split between CTAs leave
// their partial sums in p.split (slot 0 = first tile of the range, 1 = last)
// for k_adjoint_fixup, which adds them in CTA order.
template <int D, int P>
__global__ void ASH_BOUNDS(P) k_adjoint(const AdjParams p) {
  constexpr int CPS = cpair_stride(D);
  extern __shared__ float4 smem4[];
  float* sC = reinterpret_cast<float*>(smem4);
  float4* sY = reinterpret_cast<float4*>(sC + kSpotChunk * CPS);
  const int N = p.v.g.N;
  const long long u0 = p.sched.begin(blockIdx.x), u1 = p.sched.begin(blockIdx.x + 1);
  const int tf = (int)(u0 / N), tl = (int)((u1 - 1) / N);
  for (int tile = tf; tile <= tl; ++tile) {
    const int sb = (tile == tf) ? (int)(u0 - (long long)tile * N) : 0;
    const int se = (tile == tl) ? (int)(u1 - (long long)tile * N) : N;
    float2 re2[P / 2], im2[P / 2];
    adjoint_tile<D, P>(p.v, p.y, tile, sb, se, re2, im2, sC, sY);
    float2* slot = p.split + ((size_t)blockIdx.x * 2 + (tile == tf ? 0 : 1)) * kTilePix;
    adjoint_finish<P>(p.v, p.out, tile, sb == 0 && se == N, slot, re2, im2);
  }
}

// ---------------------------------------------------------------------------
// Coefficient gradient (spot-stationary): partial[b][n][d] =
//   sum over the tiles of CTA column b of Z_d(m) * Im(conj(gradE_n) f_m K_nm).
// Tiles are staged through shared memory as [pixel][dZ (D), Z (D), fr, fi].
__host__ __device__ constexpr int gradc_rec(int D) { return ((2 * D + 2) + 3) & ~3; }
__host__ __device__ constexpr size_t gradc_smem_bytes(int D) { return (size_t)kTilePix * gradc_rec(D) * 4; }

template <int D>
__global__ void __launch_bounds__(kGradThreads) k_gradc(const GradCParams p) {
  constexpr int S = kGradSpots;
  constexpr int REC = gradc_rec(D);
  extern __shared__ float4 smem4[];
  float* sP = reinterpret_cast<float*>(smem4);
  const Geometry& G = p.v.g;
  const int P = G.P, NTp = G.NT;   // pixel layout of the register-image arrays
  const int t = threadIdx.x;
  const int N = G.N;
  const int nbase = blockIdx.y * (kGradThreads * S) + t;

  float c[S][D];
  float mom[S][D];
  float2 gE[S];
  bool act[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int n = nbase + s * kGradThreads;
    act[s] = n < N;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      c[s][d] = act[s] ? __ldg(p.v.coeff + (size_t)n * D + d) : 0.0f;
      mom[s][d] = 0.0f;
    }
    gE[s] = act[s] ? __ldg(p.gradE + n) : make_float2(0.0f, 0.0f);
  }

  for (int tile = blockIdx.x; tile < G.T; tile += gridDim.x) {
    const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
    const float2* anc = p.v.anchors + (size_t)tile * D;
    __syncthreads();
    // stage the tile: pixel (tp, k) of the register-image layout -> record
    for (int e = t; e < kTilePix; e += kGradThreads) {
      const int tp = e / P, k = e % P;
      const int lane = tp & 31, wq = tp >> 5;
      const int i = tx * kTileX + lane;
      const int j = ty * kTileY + wq + (NTp / 32) * k;
      const bool valid = (i < G.nx) && (j < G.ny);
      float* rec = sP + (size_t)e * REC;
      const float* src = p.v.dz + ((size_t)tile * NTp + tp) * D * P + k;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float dzv = __ldg(src + d * P);
        const float2 a = __ldg(anc + d);
        rec[d] = dzv;
        rec[D + d] = dzv + 6.283185307179586f * (a.x + a.y);
      }
      float fr = 0.0f, fi = 0.0f;
      if (valid) {
        const float amp = __ldg(p.v.amp_img + ((size_t)tile * NTp + tp) * P + k);
        float sn, cs;
        sincosf(__ldg(p.phase + (size_t)j * G.nx + i), &sn, &cs);
        fr = amp * cs;
        fi = amp * sn;
      }
      rec[2 * D] = fr;
      rec[2 * D + 1] = fi;
    }
    // gamma = conj(gradE) exp(-i 2 pi base)
    float gr[S], gi[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      float2 a[D];
#pragma unroll
      for (int d = 0; d < D; ++d) a[d] = __ldg(anc + d);
      const float bt = base_turns<D>(c[s], a);
      const float2 r = cis_turns(-bt);
      // (gE.x - i gE.y)(r.x + i r.y)
      gr[s] = gE[s].x * r.x + gE[s].y * r.y;
      gi[s] = gE[s].x * r.y - gE[s].y * r.x;
    }
    __syncthreads();
    for (int e = 0; e < kTilePix; ++e) {
      const float* rec = sP + (size_t)e * REC;
      float z[D], za[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        z[d] = rec[d];
        za[d] = rec[D + d];
      }
      const float fr = rec[2 * D], fi = rec[2 * D + 1];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        float x = c[s][0] * z[0];
#pragma unroll
        for (int d = 1; d < D; ++d) x = fmaf(c[s][d], z[d], x);
        const float sn = __sinf(x), cs = __cosf(x);
        const float vr = fmaf(fr, cs, fi * sn);
        const float vi = fmaf(fi, cs, -fr * sn);
        const float q = fmaf(gr[s], vi, gi[s] * vr);
#pragma unroll
        for (int d = 0; d < D; ++d) mom[s][d] = fmaf(q, za[d], mom[s][d]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int n = nbase + s * kGradThreads;
    if (!act[s]) continue;
#pragma unroll
    for (int d = 0; d < D; ++d) p.partial[((size_t)blockIdx.x * N + n) * D + d] = mom[s][d];
  }
}

}  // namespace ash
