// Tensor-core variants of the transforms (see tc_common.cuh for the
// split-tf32 phase contraction and the shared-memory layout).
//
// Pixel-stationary, like the FMA kernels: a CTA of 128 threads owns a
// sub-tile of 128 x MB pixels of a 32x32 tile; thread t's pixels are
// (column t % 32, rows t / 32 + 4 k) for k = h*MB .. h*MB + MB - 1, and pixel
// block b (k = h*MB + b) is M-block b of the MMA: TMEM lane t holds thread
// t's phases. Spots stream in chunks of 16 (the MMA's N): while the tensor
// core computes chunk c + 1 into one TMEM buffer, the threads turn chunk c
// into sin/cos and complex multiply-accumulates.
#pragma once

#include "tc_common.cuh"
#include "transform_kernels.cuh"

namespace ash {

constexpr int kTcS = 16;                  // spots per MMA chunk
constexpr int kTcThreads = 128;
constexpr uint32_t kTcWaitPolls = 1u << 24;
constexpr unsigned kErrTimeout = 2u;

__host__ __device__ constexpr int tc_kp(int D) { return 3 * D <= 32 ? 32 : 64; }   // padded K
__host__ __device__ constexpr int tc_mb(int D) { return tc_kp(D) == 32 ? 4 : 2; }  // M-blocks per CTA
__host__ __device__ constexpr int tc_sub(int D) { return 8 / tc_mb(D); }           // sub-tiles per tile

// Dynamic shared memory: [1 KB alignment slack][A][B x 2][Y x 3][2 mbarriers][tmem slot].
// B (read only by the tensor core) is double-buffered: a thread stages chunk
// c + 2 only after it has itself seen the MMA of chunk c complete. The y'
// pairs are read by all threads and need three buffers: chunk c is read in
// iteration c + 1 and its buffer is rewritten in iteration c + 3, after the
// barrier of iteration c + 2.
__host__ __device__ constexpr size_t tc_smem_bytes(int D) {
  return 1024 + (size_t)tc_mb(D) * (tc_kp(D) / 32) * 16384 + 2 * (size_t)(tc_kp(D) / 32) * kTcS * 128 +
         3 * (kTcS / 2) * 32 + 64;
}

struct TcFwdParams {
  HoloView v;
  Schedule sched;            // units: (sub-tile, spot)
  const float* cz;           // [N][KP]
  const float2* rot;         // [T][N] exp(+i 2 pi base(n, tile)); the forward applies the conjugate
  const float* phase;        // user layout (kSrcPhase)
  const float2* field;       // user layout (kSrcField)
  int source;
  float* partial;            // [T * SUB * 4][2N]: row (sub-tile, warp), each entry written once
  unsigned* err;
};

struct TcAdjParams {
  HoloView v;
  Schedule sched;            // units: (sub-tile, spot), W = T * tc_sub(D) * N
  const float* cz;           // [N][KP] split coefficients [c_hi | c_hi | c_lo | 0]
  const float2* rot;         // [T][N] exp(+i 2 pi base(n, tile))
  const float2* y;           // [N]
  AdjOut out;
  float2* split;             // [G][2][kTilePix]
  unsigned* err;
};

// cz[n][k] from C: split-tf32 coefficients in K order (one thread per entry).
static __global__ void k_tc_split_coeff(const float* __restrict__ coeff, int N, int D, int KP, float* __restrict__ cz) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)N * KP) return;
  const int n = (int)(i / KP), k = (int)(i % KP);
  float v = 0.0f;
  if (k < 3 * D) {
    const int seg = k / D, d = k % D;
    const float c = coeff[(size_t)n * D + d];
    const float hi = to_tf32(c);
    v = (seg < 2) ? hi : to_tf32(c - hi);
  }
  cz[i] = v;
}

// rot[tile][n] = exp(+i 2 pi base(n, tile)): the per-(spot, tile) phase of
// the anchor pixel, reduced exactly in turns (set up once per coefficient
// matrix; the forward uses its conjugate).
static __global__ void k_tile_rotations(const float* __restrict__ coeff, const float2* __restrict__ anchors, int N,
                                        int D, int T, float2* __restrict__ rot) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)N * T) return;
  const int tile = (int)(i / N), n = (int)(i % N);
  float c[kMaxModes];
  float2 a[kMaxModes];
  for (int d = 0; d < kMaxModes; ++d) {
    c[d] = d < D ? __ldg(coeff + (size_t)n * D + d) : 0.0f;
    a[d] = d < D ? __ldg(anchors + (size_t)tile * D + d) : make_float2(0.0f, 0.0f);
  }
  // modes beyond D have c = 0 and contribute exactly 0 turns
  rot[i] = cis_turns(base_turns<kMaxModes>(c, a));
}

template <int D>
__global__ void __launch_bounds__(kTcThreads, 3) k_tc_adjoint(const TcAdjParams p) {
  constexpr int KP = tc_kp(D), MB = tc_mb(D), NA = KP / 32, SUB = tc_sub(D), S = kTcS;
  constexpr uint32_t NCOLS = 2 * MB * S;   // two TMEM buffers of MB x S fp32 columns
  constexpr uint32_t IDESC = umma_idesc_tf32(128, S);
  constexpr int BV = NA * S * 8 / kTcThreads;   // 16-byte pieces of a B chunk per thread
  static_assert(BV * kTcThreads == NA * S * 8, "B chunk must split evenly over the CTA");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* sA = reinterpret_cast<float*>(base);                        // [MB][NA][128 x 32]
  float* sB = sA + MB * NA * 4096;                                   // [2][NA][S x 32]
  float* sY = sB + 2 * NA * S * 32;                                  // [3][S/2][8]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sY + 3 * (S / 2) * 8);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == 0) tmem_alloc(tslot, NCOLS);
  if (t == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = (uint32_t)(w * 32) << 16;
  uint32_t parity = 0;
  bool ok = true;

  const Geometry& G = p.v.g;
  const int N = G.N;
  const long long u0 = p.sched.begin(blockIdx.x), u1 = p.sched.begin(blockIdx.x + 1);
  const int sf = (int)(u0 / N), sl = (int)((u1 - 1) / N);

  // chunk staging in two halves: fetch() issues the global loads into
  // registers, put() stores them (B rows to sB[buf], y' pairs to sY[ybuf])
  float4 bv[BV];
  float2 yv = make_float2(0.0f, 0.0f), rv = make_float2(0.0f, 0.0f);
  auto fetch = [&](int tile, int n0, int se) {
#pragma unroll
    for (int q = 0; q < BV; ++q) {
      const int e = t + q * kTcThreads;
      const int atom = e / (S * 8), r = (e / 8) % S, j = e % 8;
      const int n = n0 + r;
      bv[q] = n < se ? __ldg(reinterpret_cast<const float4*>(p.cz + (size_t)n * KP + atom * 32 + 4 * j))
                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    if (t < S) {
      const int n = n0 + t;
      yv = n < se ? __ldg(p.y + n) : make_float2(0.0f, 0.0f);
      rv = n < se ? __ldg(p.rot + (size_t)tile * N + n) : make_float2(0.0f, 0.0f);
    }
  };
  auto put = [&](int buf, int ybuf) {
#pragma unroll
    for (int q = 0; q < BV; ++q) {
      const int e = t + q * kTcThreads;
      const int atom = e / (S * 8), r = (e / 8) % S, j = e % 8;
      *reinterpret_cast<float4*>(sB + (buf * NA + atom) * (S * 32) + swz128(r, 4 * j)) = bv[q];
    }
    if (t < S) {
      const float yr = yv.x * rv.x - yv.y * rv.y;
      const float yi = yv.x * rv.y + yv.y * rv.x;
      float* yq = sY + (ybuf * (S / 2) + (t >> 1)) * 8;
      yq[(t & 1)] = yr;
      yq[2 + (t & 1)] = yi;
      yq[4 + (t & 1)] = -yi;
      yq[6 + (t & 1)] = 0.0f;
    }
    fence_async_smem();
  };

  for (int st = sf; st <= sl; ++st) {
    const int tile = st / SUB, h = st % SUB;
    const int sb = (st == sf) ? (int)(u0 - (long long)st * N) : 0;
    const int se = (st == sl) ? (int)(u1 - (long long)st * N) : N;
    const int nch = (se - sb + S - 1) / S;

    fetch(tile, sb, se);
    // A: this thread's MB pixels as split-tf32 rows of the MB M-blocks
    {
      float z[D][MB];
      const float* src = p.v.dz + ((size_t)tile * 128 + t) * D * 8 + h * MB;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if constexpr (MB == 4) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(src + d * 8));
          z[d][0] = q.x; z[d][1] = q.y; z[d][2] = q.z; z[d][3] = q.w;
        } else {
          const float2 q = __ldg(reinterpret_cast<const float2*>(src + d * 8));
          z[d][0] = q.x; z[d][MB - 1] = q.y;
        }
      }
#pragma unroll
      for (int b = 0; b < MB; ++b) {
        float row[KP];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float hi = to_tf32(z[d][b]);
          row[d] = hi;
          row[D + d] = to_tf32(z[d][b] - hi);
          row[2 * D + d] = hi;
        }
#pragma unroll
        for (int k = 3 * D; k < KP; ++k) row[k] = 0.0f;
#pragma unroll
        for (int j = 0; j < KP / 4; ++j) {
          const int atom = (4 * j) / 32, kk = (4 * j) % 32;
          *reinterpret_cast<float4*>(sA + (b * NA + atom) * 4096 + swz128(t, kk)) =
              make_float4(row[4 * j], row[4 * j + 1], row[4 * j + 2], row[4 * j + 3]);
        }
      }
    }
    put(0, 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    float2 re2[MB], im2[MB];
#pragma unroll
    for (int b = 0; b < MB; ++b) re2[b] = im2[b] = make_float2(0.0f, 0.0f);

    for (int c = 0; c <= nch; ++c) {
      // B(c) and y'(c) are in shared memory (previous barrier): start MMA(c)
      if (c < nch && t == 0) {
        const int buf = c & 1;
#pragma unroll
        for (int b = 0; b < MB; ++b) {
#pragma unroll
          for (int ks = 0; ks < KP / 8; ++ks) {
            const int atom = ks / 4, koff = (ks % 4) * 32;
            const uint64_t ad = umma_desc(smem_u32(sA + (b * NA + atom) * 4096) + koff);
            const uint64_t bd = umma_desc(smem_u32(sB + (buf * NA + atom) * (S * 32)) + koff);
            umma_tf32(tmem + (uint32_t)(buf * MB * S + b * S), ad, bd, IDESC, ks > 0 ? 1u : 0u);
          }
        }
        umma_commit(&mbar[buf]);
      }
      // loads for chunk c + 1 in flight while chunk c - 1 is consumed
      if (c + 1 < nch) fetch(tile, sb + (c + 1) * S, se);
      if (c >= 1) {
        const int buf = (c - 1) & 1, ybuf = (c - 1) % 3;
        ok = mbar_wait(&mbar[buf], (parity >> buf) & 1u, kTcWaitPolls) && ok;
        parity ^= 1u << buf;
        tc_fence_after();
        float2 yr2[S / 2], yi2[S / 2], nyi2[S / 2];
#pragma unroll
        for (int q = 0; q < S / 2; ++q) {
          const float4 a = *reinterpret_cast<const float4*>(sY + (ybuf * (S / 2) + q) * 8);
          const float4 bq = *reinterpret_cast<const float4*>(sY + (ybuf * (S / 2) + q) * 8 + 4);
          yr2[q] = make_float2(a.x, a.y);
          yi2[q] = make_float2(a.z, a.w);
          nyi2[q] = make_float2(bq.x, bq.y);
        }
        uint32_t xr[MB][16];
#pragma unroll
        for (int b = 0; b < MB; ++b) tmem_ld16_nowait(tmem + tlane + (uint32_t)(buf * MB * S + b * S), xr[b]);
        tmem_wait();
#pragma unroll
        for (int b = 0; b < MB; ++b) {
#pragma unroll
          for (int q = 0; q < S / 2; ++q) {
            float2 sn, cs;
            sincos2(make_float2(__uint_as_float(xr[b][2 * q]), __uint_as_float(xr[b][2 * q + 1])), sn, cs);
            re2[b] = fma2(yr2[q], cs, re2[b]);
            re2[b] = fma2(nyi2[q], sn, re2[b]);
            im2[b] = fma2(yi2[q], cs, im2[b]);
            im2[b] = fma2(yr2[q], sn, im2[b]);
          }
        }
      }
      // chunk c + 1 into buffer (c + 1) & 1: its previous user, MMA(c - 1), is
      // complete (this thread waited for it just above)
      if (c + 1 < nch) put((c + 1) & 1, (c + 1) % 3);
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }

    // epilogue (whole spot range owned) or partial sums for the fix-up
    const bool full = (sb == 0 && se == N);
    const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
    const int i = tx * kTileX + lane;
    float2* slot = p.split + ((size_t)blockIdx.x * 2 + (st == sf ? 0 : 1)) * kTilePix;
#pragma unroll
    for (int b = 0; b < MB; ++b) {
      const float gr = re2[b].x + re2[b].y, gi = im2[b].x + im2[b].y;
      if (full) {
        const int k = h * MB + b;
        const int j = ty * kTileY + w + 4 * k;
        if (i < G.nx && j < G.ny) {
          const float a = (p.out.epilogue & kEpiGradPhase) ? __ldg(p.v.amp_img + ((size_t)tile * 128 + t) * 8 + k) : 0.0f;
          adjoint_epilogue(p.out, (size_t)j * G.nx + i, gr, gi, a);
        }
      } else {
        slot[b * kTcThreads + t] = make_float2(gr, gi);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem, NCOLS);
  if (!ok && t == 0) atomicOr(p.err, kErrTimeout);
}

// Forward: partial[(sub-tile, warp)][2n..2n+1] = exp(-i 2 pi base(n, tile))
// x sum over the warp's pixels of the sub-tile of f_m exp(-i dZ_m . C_n).
template <int D>
__global__ void __launch_bounds__(kTcThreads, 3) k_tc_forward(const TcFwdParams p) {
  constexpr int KP = tc_kp(D), MB = tc_mb(D), NA = KP / 32, SUB = tc_sub(D), S = kTcS;
  constexpr uint32_t NCOLS = 2 * MB * S;
  constexpr uint32_t IDESC = umma_idesc_tf32(128, S);
  constexpr int BV = NA * S * 8 / kTcThreads;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* sA = reinterpret_cast<float*>(base);
  float* sB = sA + MB * NA * 4096;
  float* sY = sB + 2 * NA * S * 32;                                  // unused by the forward
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sY + 3 * (S / 2) * 8);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (w == 0) tmem_alloc(tslot, NCOLS);
  if (t == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = (uint32_t)(w * 32) << 16;
  uint32_t parity = 0;
  bool ok = true;

  const Geometry& G = p.v.g;
  const int N = G.N;
  const long long u0 = p.sched.begin(blockIdx.x), u1 = p.sched.begin(blockIdx.x + 1);
  const int sf = (int)(u0 / N), sl = (int)((u1 - 1) / N);

  float4 bv[BV];
  float2 rot_next = make_float2(0.0f, 0.0f), rot_cur = make_float2(0.0f, 0.0f);
  // loads of chunk (n0 .. n0 + S) issued one iteration ahead of their use:
  // B rows (split coefficients) and this lane's spot rotation
  auto fetch = [&](int tile, int n0, int se) {
#pragma unroll
    for (int q = 0; q < BV; ++q) {
      const int e = t + q * kTcThreads;
      const int atom = e / (S * 8), r = (e / 8) % S, j = e % 8;
      const int n = n0 + r;
      bv[q] = n < se ? __ldg(reinterpret_cast<const float4*>(p.cz + (size_t)n * KP + atom * 32 + 4 * j))
                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    const int n = n0 + (lane >> 1);
    rot_next = n < se ? __ldg(p.rot + (size_t)tile * N + n) : make_float2(1.0f, 0.0f);
  };
  auto put = [&](int buf) {
#pragma unroll
    for (int q = 0; q < BV; ++q) {
      const int e = t + q * kTcThreads;
      const int atom = e / (S * 8), r = (e / 8) % S, j = e % 8;
      *reinterpret_cast<float4*>(sB + (buf * NA + atom) * (S * 32) + swz128(r, 4 * j)) = bv[q];
    }
    fence_async_smem();
  };

  for (int st = sf; st <= sl; ++st) {
    const int tile = st / SUB, h = st % SUB;
    const int sb = (st == sf) ? (int)(u0 - (long long)st * N) : 0;
    const int se = (st == sl) ? (int)(u1 - (long long)st * N) : N;
    const int nch = (se - sb + S - 1) / S;
    const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
    const int i = tx * kTileX + lane;

    fetch(tile, sb, se);
    // A rows and this thread's nearfield values (duplicated for packed FMAs)
    float2 frr[MB], fii[MB], nfrr[MB];
    {
      float z[D][MB];
      const float* src = p.v.dz + ((size_t)tile * 128 + t) * D * 8 + h * MB;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if constexpr (MB == 4) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(src + d * 8));
          z[d][0] = q.x; z[d][1] = q.y; z[d][2] = q.z; z[d][3] = q.w;
        } else {
          const float2 q = __ldg(reinterpret_cast<const float2*>(src + d * 8));
          z[d][0] = q.x; z[d][MB - 1] = q.y;
        }
      }
#pragma unroll
      for (int b = 0; b < MB; ++b) {
        float row[KP];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float hi = to_tf32(z[d][b]);
          row[d] = hi;
          row[D + d] = to_tf32(z[d][b] - hi);
          row[2 * D + d] = hi;
        }
#pragma unroll
        for (int k = 3 * D; k < KP; ++k) row[k] = 0.0f;
#pragma unroll
        for (int j = 0; j < KP / 4; ++j) {
          const int atom = (4 * j) / 32, kk = (4 * j) % 32;
          *reinterpret_cast<float4*>(sA + (b * NA + atom) * 4096 + swz128(t, kk)) =
              make_float4(row[4 * j], row[4 * j + 1], row[4 * j + 2], row[4 * j + 3]);
        }
        const int k = h * MB + b;
        const int j = ty * kTileY + w + 4 * k;
        const bool valid = (i < G.nx) && (j < G.ny);
        const size_t m = (size_t)j * G.nx + i;
        float fr = 0.0f, fi = 0.0f;
        if (valid) {
          if (p.source == kSrcPhase) {
            const float a = __ldg(p.v.amp_img + ((size_t)tile * 128 + t) * 8 + k);
            float sn, cs;
            sincosf(__ldg(p.phase + m), &sn, &cs);
            fr = a * cs;
            fi = a * sn;
          } else {
            const float2 f = __ldg(p.field + m);
            fr = f.x;
            fi = f.y;
          }
        }
        frr[b] = make_float2(fr, fr);
        fii[b] = make_float2(fi, fi);
        nfrr[b] = make_float2(-fr, -fr);
      }
    }
    put(0);
    rot_cur = rot_next;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    float* prow = p.partial + ((size_t)st * 4 + w) * 2 * N;

    for (int c = 0; c <= nch; ++c) {
      if (c < nch && t == 0) {
        const int buf = c & 1;
#pragma unroll
        for (int b = 0; b < MB; ++b) {
#pragma unroll
          for (int ks = 0; ks < KP / 8; ++ks) {
            const int atom = ks / 4, koff = (ks % 4) * 32;
            const uint64_t ad = umma_desc(smem_u32(sA + (b * NA + atom) * 4096) + koff);
            const uint64_t bd = umma_desc(smem_u32(sB + (buf * NA + atom) * (S * 32)) + koff);
            umma_tf32(tmem + (uint32_t)(buf * MB * S + b * S), ad, bd, IDESC, ks > 0 ? 1u : 0u);
          }
        }
        umma_commit(&mbar[buf]);
      }
      // rot_cur belongs to chunk c - 1 (consumed below); chunk c's is in rot_next
      const float2 rot_use = rot_cur;
      rot_cur = rot_next;
      if (c + 1 < nch) fetch(tile, sb + (c + 1) * S, se);
      if (c >= 1) {
        const int buf = (c - 1) & 1, n0 = sb + (c - 1) * S;
        ok = mbar_wait(&mbar[buf], (parity >> buf) & 1u, kTcWaitPolls) && ok;
        parity ^= 1u << buf;
        tc_fence_after();
        uint32_t xr[MB][16];
#pragma unroll
        for (int b = 0; b < MB; ++b) tmem_ld16_nowait(tmem + tlane + (uint32_t)(buf * MB * S + b * S), xr[b]);
        tmem_wait();
        float2 re2[S / 2], im2[S / 2];
#pragma unroll
        for (int q = 0; q < S / 2; ++q) {
          re2[q] = im2[q] = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int b = 0; b < MB; ++b) {
            float2 sn, cs;
            sincos2(make_float2(__uint_as_float(xr[b][2 * q]), __uint_as_float(xr[b][2 * q + 1])), sn, cs);
            // f exp(-i x) = (fr cs + fi sn) + i (fi cs - fr sn)
            re2[q] = fma2(frr[b], cs, re2[q]);
            re2[q] = fma2(fii[b], sn, re2[q]);
            im2[q] = fma2(fii[b], cs, im2[q]);
            im2[q] = fma2(nfrr[b], sn, im2[q]);
          }
        }
        float acc[32];
#pragma unroll
        for (int q = 0; q < S / 2; ++q) {
          acc[4 * q] = re2[q].x;
          acc[4 * q + 1] = im2[q].x;
          acc[4 * q + 2] = re2[q].y;
          acc[4 * q + 3] = im2[q].y;
        }
        const float v = warp_transpose_reduce32(acc, lane);
        const float other = __shfl_xor_sync(kFull, v, 1);
        const bool is_im = (lane & 1) != 0;
        const int n = n0 + (lane >> 1);
        if (n < se) {
          const float re = is_im ? other : v;
          const float im = is_im ? v : other;
          // exp(+i 2 pi base) was loaded one iteration ago: multiply by its conjugate
          prow[2 * n + (lane & 1)] = is_im ? fmaf(im, rot_use.x, -re * rot_use.y) : fmaf(re, rot_use.x, im * rot_use.y);
        }
      }
      if (c + 1 < nch) put((c + 1) & 1);
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tmem, NCOLS);
  if (!ok && t == 0) atomicOr(p.err, kErrTimeout);
}

// Finishes sub-tiles split between CTAs of k_tc_adjoint (fixed CTA order).
// One CTA of 128 threads per sub-tile; sub-tiles owned by one CTA return.
static __global__ void k_tc_adjoint_fixup(const TcAdjParams p, int MB) {
  const Geometry& G = p.v.g;
  const int SUB = 8 / MB;
  const int st = blockIdx.x, t = threadIdx.x;
  const long long u_lo = (long long)st * G.N, u_hi = u_lo + G.N - 1;
  const int b_lo = p.sched.owner(u_lo), b_hi = p.sched.owner(u_hi);
  if (b_lo == b_hi) return;
  const int tile = st / SUB, h = st % SUB;
  const int tx = tile % G.tiles_x, ty = tile / G.tiles_x;
  const int i = tx * kTileX + (t & 31);
  for (int b = 0; b < MB; ++b) {
    float gr = 0.0f, gi = 0.0f;
    for (int cb = b_lo; cb <= b_hi; ++cb) {
      const int slot = (p.sched.begin(cb) >= u_lo) ? 0 : 1;
      const float2 v = p.split[((size_t)cb * 2 + slot) * kTilePix + b * kTcThreads + t];
      gr += v.x;
      gi += v.y;
    }
    const int k = h * MB + b;
    const int j = ty * kTileY + (t >> 5) + 4 * k;
    if (i >= G.nx || j >= G.ny) continue;
    const float a = (p.out.epilogue & kEpiGradPhase) ? p.v.amp_img[((size_t)tile * 128 + t) * 8 + k] : 0.0f;
    adjoint_epilogue(p.out, (size_t)j * G.nx + i, gr, gi, a);
  }
}

}  // namespace ash
