// Tensor-core transforms (see tc_common.cuh for the split-tf32 phase
// contraction and the operand layout, tc_launch.h for the parameter blocks).
//
// Both transforms contract 128 rows of one kind with 64 of the other per MMA
// (M = 128, N = 64): the tensor core's cost per instruction is flat up to
// N = 64, so wide chunks keep it far below the MUFU time.
//
//  * adjoint, pixel-stationary: A = the split basis rows of 128 pixels (a
//    "group": rows 4h .. 4h + 3 of a 32x32 tile), B = 64 spots; thread t owns
//    pixel t and accumulates g over all spots of its range;
//  * forward, spot-stationary: A = 128 spots, B = 64 pixels (a "chunk": half
//    a group); thread t owns spot t and accumulates E over its pixels, so no
//    cross-thread reduction is needed.
//
// Operands are laid out in HBM exactly as the MMA reads them from shared
// memory (pre-split, pre-swizzled), so one thread moves each chunk with the
// bulk-copy engine (cp.async.bulk) into a ring of shared-memory slots
// tracked by mbarriers. Two TMEM buffers of 64 fp32 columns alternate: each
// warp copies a chunk's phases out of TMEM, arrives on a shared counter and
// goes on to the sincos and the complex multiply-accumulate; the warp that
// arrives last refills the rings and issues the next MMAs: in the forward
// two chunks ahead, into the buffer just freed; in the adjoint one chunk
// ahead (its shared memory holds two spot-row slots, so that four CTAs fit
// on an SM). No CTA-wide barrier is taken in the main loop. The
// producer steps of consecutive chunks cannot overlap: the last arrival for
// chunk c comes after every warp's arrival for c, and the warp that ran the
// producer step of c - 1 arrives for c only after finishing it (its release
// on the counter publishes the producer state to the next producer).
//
// Per-tile anchor phases: for a pixel m of tile tau,
//   C_n . Z_m = 2 pi base(n, tau) + C_n . dZ_m,
// with base reduced exactly in turns once per (spot, tile) (rot[tau][n] =
// exp(+i 2 pi base)); the tensor core computes C_n . dZ_m only.
#pragma once

#include "common.cuh"
#include "tc_common.cuh"
#include "tc_launch.h"

namespace ash {

// Adjoint shared memory: 2 A slots (groups), 2 B slots (spot chunks), y' per
// warp (four CTAs per SM for NA = 1).
template <int NA>
struct TcAdjShape {
  static constexpr int NB = 2;
  static constexpr uint32_t A_BYTES = NA * 16384, B_BYTES = NA * 8192;
  static constexpr uint32_t Y_BYTES = 4 * 32 * 16;
  static constexpr int NBARS = 4 + NB;
  // [alignment slack][A x 2][B ring][y'][barriers][armed counts][counter][TMEM slot][producer state]
  static constexpr size_t SMEM = 1024 + 2 * A_BYTES + NB * B_BYTES + Y_BYTES + NBARS * 12 + 8 + 16;
  static constexpr size_t TSLOT = 2 * A_BYTES + NB * B_BYTES + Y_BYTES + NBARS * 12 + 8;   // from the aligned base
};

// Forward shared memory: 1 A slot (spot block), a ring of B slots (64 pixel
// rows, read by the tensor core) and a ring of f slots (the 64 pixels'
// nearfield, read by the threads). Each copy is issued several chunks
// before its use, which keeps HBM latency hidden even where a chunk's
// arithmetic is short (a partial last spot block).
template <int NA>
struct TcFwdShape {
  // KF = 5 (an 8-slot f ring) measured 1-2 % faster than 3, 4, 7 or 10
  static constexpr int NBB = NA == 1 ? 4 : 3, KF = 5, NF = KF + 3;
  static constexpr uint32_t A_BYTES = NA * 16384, B_BYTES = NA * 8192, F_BYTES = 512;
  static constexpr int NBARS = 3 + NBB + NF;
  // [alignment slack][A][B ring][f ring][barriers][armed counts][counter][TMEM slot][producer state]
  static constexpr size_t SMEM = 1024 + A_BYTES + NBB * B_BYTES + NF * F_BYTES + NBARS * 12 + 8 + 32;
  static constexpr size_t TSLOT = A_BYTES + NBB * B_BYTES + NF * F_BYTES + NBARS * 12 + 8;
};

// --- operand images ---------------------------------------------------------

// zs from the register-image basis dz: one thread per (chunk, row).
static __global__ void k_tc_build_zs(const Geometry G, const TcLayout L, const float* __restrict__ dz,
                                     float* __restrict__ zs) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)G.T * kTcChunksPerTile * kTcChunk) return;
  const long long qc = e / kTcChunk;
  const int r = (int)(e % kTcChunk), D = G.D;
  const TcPixel px = tc_pixel(G, qc, r);
  const bool in = px.i < G.nx && px.j < G.ny;
  int ia, ja;
  tile_anchor(G, px.tile, ia, ja);
  const int tpx = px.img / G.P, k = px.img % G.P;
  float* dst = zs + (size_t)qc * L.NA * 2048;
  for (int a = 0; a < L.NA; ++a)
    for (int kk = 0; kk < 32; ++kk) {
      int kind, mode;
      tc_slot(L, 32 * a + kk, kind, mode);
      float v = 0.0f;
      if (kind >= 0 && kind < 3) {
        const float z = dz[((size_t)tpx * D + mode) * G.P + k];
        const float hi = to_tf32(z);
        v = kind == 1 ? to_tf32(z - hi) : hi;   // [hi | lo | hi]
      } else if (kind == 3 && in) {
        v = (float)(px.i - ia);                 // exact integer offsets
      } else if (kind == 4 && in) {
        v = (float)(px.j - ja);
      }
      dst[a * 2048 + swz128(r, kk)] = v;
    }
}

// czs from the coefficients, in turns (C / 2 pi, so that the MMA gives the
// local phase in turns): one thread per (spot chunk, row); rows >= N are 0.
// The two chunks after the nc64 main ones hold the last 128-spot block with
// its first 128 / rep spots repeated rep times.
constexpr double kInv2PiD = 0.15915494309189533576888376337251;
static __global__ void k_tc_build_czs(const float* __restrict__ coeff, int N, const TcLayout L, int nc64, int rep,
                                      float* __restrict__ czs) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)(nc64 + 2) * kTcChunk) return;
  const int jc = (int)(e / kTcChunk), r = (int)(e % kTcChunk), D = L.D;
  int n = jc * kTcChunk + r;
  if (jc >= nc64) n = (nc64 - 2) * kTcChunk + ((jc - nc64) * kTcChunk + r) % (kTcRows / rep);
  float* dst = czs + (size_t)jc * L.NA * 2048;
  for (int a = 0; a < L.NA; ++a)
    for (int kk = 0; kk < 32; ++kk) {
      int kind, mode;
      tc_slot(L, 32 * a + kk, kind, mode);
      float v = 0.0f;
      if (kind >= 0 && n < N) {
        if (kind < 3) {
          // in turns: the products give the local phase / 2 pi
          const double c = (double)coeff[(size_t)n * D + mode] * kInv2PiD;
          const float hi = to_tf32((float)c);
          v = kind == 2 ? to_tf32((float)(c - (double)hi)) : hi;   // [hi | hi | lo]
        } else {
          // turns per pixel, split into tf32 pieces (piece `mode`)
          const double cr = (double)coeff[(size_t)n * D + (kind == 3 ? L.tx : L.ty)] / (double)L.R * kInv2PiD;
          double rest = cr;
          for (int q = 0; q <= mode; ++q) {
            const float piece = to_tf32((float)rest);
            v = piece;
            rest -= (double)piece;
          }
        }
      }
      dst[a * 2048 + swz128(r, kk)] = v;
    }
}

// A phase in turns, reduced to [-1/2, 1/2] (the nearfield image's phases
// stay small, so that phi - x keeps the accuracy of x).
__device__ __forceinline__ float turns_of_phase(float ph) {
  const float t = ph * 0.15915494309189535f;
  return t - rintf(t);
}

// Nearfield in tc layout, as amplitude and phase in turns: f = A exp(i 2 pi
// phi) from a phase or from a complex field (A = |f|, phi = arg f / 2 pi),
// both in user layout; pixels outside the grid are 0. Chunk pixel pair p
// holds (A_2p, A_2p+1, phi_2p, phi_2p+1).
static __global__ void k_tc_field_img(const Geometry G, const float* __restrict__ amp_img,
                                      const float* __restrict__ phase, const float2* __restrict__ field,
                                      float* __restrict__ fimg) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)G.T * kTilePix) return;
  const long long qc = e / kTcChunk;
  const int r = (int)(e % kTcChunk);
  const TcPixel px = tc_pixel(G, qc, r);
  float a = 0.0f, ph = 0.0f;
  if (px.i < G.nx && px.j < G.ny) {
    const size_t m = (size_t)px.j * G.nx + px.i;
    if (phase) {
      a = amp_img[px.img];
      ph = turns_of_phase(phase[m]);
    } else {
      const float2 f = field[m];
      a = hypotf(f.x, f.y);
      ph = (f.x == 0.0f && f.y == 0.0f) ? 0.0f : atan2f(f.y, f.x) * 0.15915494309189535f;
    }
  }
  float* q = fimg + ((size_t)qc * 32 + (r >> 1)) * 4;
  q[r & 1] = a;
  q[2 + (r & 1)] = ph;
}

// rot[tile][n] = exp(+i 2 pi base(n, tile)): the per-(spot, tile) phase of
// the anchor pixel, reduced exactly in turns.
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

// --- pieces shared by the two kernels ------------------------------------------

template <bool V>
struct BoolTag {
  static constexpr bool value = V;
};

// D[tmem] = A[128 rows] . B[64 rows]^T over KP = 32 NA, issued by one thread.
template <int NA>
__device__ __forceinline__ void tc_mma_chunk(uint32_t tmem_cols, const float* sA, const float* sB, uint64_t* done) {
  constexpr uint32_t IDESC = umma_idesc_tf32(kTcRows, kTcChunk);
#pragma unroll
  for (int ks = 0; ks < 4 * NA; ++ks) {
    const int atom = ks / 4, koff = (ks % 4) * 32;
    const uint64_t ad = umma_desc(smem_u32(sA + atom * 4096) + koff);
    const uint64_t bd = umma_desc(smem_u32(sB + atom * 2048) + koff);
    umma_tf32(tmem_cols, ad, bd, IDESC, ks > 0 ? 1u : 0u);
  }
  umma_commit(done);
}

// Bulk copy of 128 operand rows (two consecutive 64-row chunk images) into
// a [NA][128][32] slot.
template <int NA>
__device__ __forceinline__ void tc_copy_rows128(float* dst, const float* src, uint64_t* bar) {
  if constexpr (NA == 1) {
    bulk_g2s(dst, src, 16384, bar);
  } else {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      bulk_g2s(dst + a * 4096, src + a * 2048, 8192, bar);
      bulk_g2s(dst + a * 4096 + 2048, src + NA * 2048 + a * 2048, 8192, bar);
    }
  }
}

// 16-column groups [q_lo, q_hi) of this warp's 32 TMEM lanes, one wait.
__device__ __forceinline__ void tc_load_cols(uint32_t taddr, int q_lo, int q_hi, uint32_t (&x)[4][16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q >= q_lo && q < q_hi) tmem_ld16_nowait(taddr + 16 * q, x[q]);
  tmem_wait();
}

// Bounded wait for the last armed phase of each barrier, so that no copy or
// MMA is still in flight when the CTA frees its memory (all of them have
// completed already unless a wait timed out).
__device__ __forceinline__ void tc_drain(uint64_t* bars, const uint32_t* armed, int nbars) {
  for (int k = 0; k < nbars; ++k)
    if (armed[k] > 0) mbar_wait(&bars[k], (armed[k] - 1) & 1u, kTcWaitPolls);
}

__device__ __forceinline__ uint8_t* tc_smem_base(uint8_t* raw) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
}

// Two TMEM buffers of 64 fp32 columns for the CTA's lifetime (warp 0).
__device__ __forceinline__ uint32_t tc_tmem_alloc(uint32_t* slot) {
  if ((threadIdx.x >> 5) == 0) tmem_alloc(slot, 2 * kTcChunk);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *slot;
}

__device__ __forceinline__ void tc_tmem_free(uint32_t tmem) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, 2 * kTcChunk);
}

// Start of one unit range: fresh barriers (the previous range's, if any, are
// invalidated first), counters at zero, then a CTA barrier.
__device__ __forceinline__ void tc_range_begin(uint64_t* bars, uint32_t* armed, uint32_t* cnt, int nbars, bool first) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < nbars; ++k) {
      if (!first) mbar_inval(&bars[k]);
      mbar_init(&bars[k], 1);
      armed[k] = 0;
    }
    cnt[0] = cnt[1] = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// End of a range: every thread is done, every copy and MMA has landed.
__device__ __forceinline__ void tc_range_end(uint64_t* bars, const uint32_t* armed, int nbars, bool drained = false) {
  if (!drained) {
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) tc_drain(bars, armed, nbars);
  }
  __syncthreads();
}

// Adjoint output of row r of chunk qc (in the pixel's user-layout slot and,
// for kEpiFimg, in the tc-layout nearfield f = A exp(i arg g) as (A, arg g / 2 pi)).
__device__ __forceinline__ void tc_adjoint_epilogue(const TcAdjParams& p, long long qc, int r, float gr, float gi) {
  const Geometry& G = p.g;
  const TcPixel px = tc_pixel(G, qc, r);
  if (px.i >= G.nx || px.j >= G.ny) return;
  const bool need_a = (p.out.epilogue & (kEpiGradPhase | kEpiFimg)) != 0;
  const float a = need_a ? __ldg(p.amp_img + px.img) : 0.0f;
  adjoint_epilogue(p.out, (size_t)px.j * G.nx + px.i, gr, gi, a);
  if (p.out.epilogue & kEpiFimg) {
    const float ph = (gr == 0.0f && gi == 0.0f) ? 0.0f : atan2f(gi, gr) * 0.15915494309189535f;
    float* q = reinterpret_cast<float*>(p.fimg + (size_t)qc * 32 + (r >> 1));
    q[r & 1] = a;
    q[2 + (r & 1)] = ph;
  }
}

// --- adjoint ------------------------------------------------------------------

// g_m = sum_n y_n exp(+i C_n . Z_m) for the pixels of this CTA's (group,
// spot chunk) range; groups whose spots are split between CTAs go through
// `split` and k_tc_adjoint_fixup.
//
// Producer schedule: the warp releasing chunk c last issues the MMA of
// chunk c + 2 into the TMEM buffer just released (it completes while the
// warps work through chunks c and c + 1); the warp releasing it first loads
// B of chunk c + NB into the slot MMA(c) has freed, and A of group s + 2
// into the slot of group s once c is s's last chunk. The first release of
// a chunk comes well before its last (the warps drift apart by up to about
// two chunks), so chunk c + 2's B is in place when its MMA is issued with a
// two-slot B ring. (Measured at 1024^2, N = 400: 274 us against 280 with
// the MMA one chunk ahead.)
template <int NA, bool REDUCE = true>
__device__ __forceinline__ void tc_adjoint_range(const TcAdjParams& p, long long u0, long long u1, int cta,
                                                 uint8_t* base, uint32_t tmem, bool first_range) {
  using S = TcAdjShape<NA>;
  constexpr int NB = S::NB, NBARS = S::NBARS;
  float* sA = reinterpret_cast<float*>(base);                      // [2][NA][128][32]
  float* sB = sA + 2 * NA * 4096;                                  // [NB][NA][64][32]
  float4* sY = reinterpret_cast<float4*>(sB + NB * NA * 2048);     // [4 warps][32 spot pairs]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sY + 4 * 32);       // full[2] | bfull[NB] | afull[2]
  uint64_t* full = bars;
  uint64_t* bfull = bars + 2;
  uint64_t* afull = bars + 2 + NB;
  uint32_t* armed = reinterpret_cast<uint32_t*>(bars + NBARS);     // phases armed per barrier
  uint32_t* cnt = armed + NBARS;                                   // [2] arrivals per TMEM buffer
  uint32_t* tslot = cnt + 2;
  int* pst = reinterpret_cast<int*>(tslot + 1);                    // next MMA: chunk, group, spot chunk

  (void)tslot;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const Geometry& G = p.g;
  const int N = G.N;
  const int nch = (N + kTcChunk - 1) / kTcChunk;
  const int nc = (int)(u1 - u0);
  // chunk c of this range is spot chunk j of group s; (s, j) advance
  // incrementally (no 64-bit division per chunk)
  const int s0 = (int)(u0 / nch), j0 = (int)(u0 % nch);
  const int s_last = nc > 0 ? (int)((u1 - 1) / nch) : s0;

  tc_range_begin(bars, armed, cnt, NBARS, first_range);
  const uint32_t tlane = (uint32_t)(w * 32) << 16;
  bool ok = true;

  // --- producer steps (one thread at a time) ---
  auto load_a = [&](int s) {
    const int slot = (s - s0) & 1;
    mbar_expect_tx(&afull[slot], S::A_BYTES);
    ++armed[2 + NB + slot];
    tc_copy_rows128<NA>(sA + slot * NA * 4096, p.zs + (size_t)(2 * s) * NA * 2048, &afull[slot]);
  };
  auto load_b = [&](int c, int j) {
    const int slot = c % NB;
    mbar_expect_tx(&bfull[slot], S::B_BYTES);
    ++armed[2 + slot];
    bulk_g2s(sB + slot * NA * 2048, p.czs + (size_t)j * NA * 2048, S::B_BYTES, &bfull[slot]);
  };
  auto issue_upto = [&](int upto) -> bool {
    bool r = true;
    int k = pst[0], s = pst[1], j = pst[2];
    for (; k <= upto && k < nc; ++k) {
      const int ls = s - s0;
      r = mbar_wait(&bfull[k % NB], (uint32_t)((k / NB) & 1), kTcWaitPolls) && r;
      if (k == 0 || j == 0) r = mbar_wait(&afull[ls & 1], (uint32_t)((ls >> 1) & 1), kTcWaitPolls) && r;
      tc_fence_after();
      ++armed[k & 1];
      tc_mma_chunk<NA>(tmem + (uint32_t)((k & 1) * kTcChunk), sA + (ls & 1) * NA * 4096, sB + (k % NB) * NA * 2048,
                       &full[k & 1]);
      if (++j == nch) {
        j = 0;
        ++s;
      }
    }
    pst[0] = k;
    pst[1] = s;
    pst[2] = j;
    return r;
  };

  int jb = j0;                       // spot chunk of chunk c + NB (the next B to load)
  for (int k = 0; k < NB; ++k)
    if (++jb == nch) jb = 0;
  if (t == 0 && nc > 0) {
    pst[0] = 0;
    pst[1] = s0;
    pst[2] = j0;
    load_a(s0);
    if (s0 + 1 <= s_last) load_a(s0 + 1);
    for (int c = 0, j = j0; c < NB && c < nc; ++c, j = (j + 1 == nch ? 0 : j + 1)) load_b(c, j);
    ok = issue_upto(1);
  }

  float4* yw = sY + w * 32;   // this warp's (yr, yr', yi, yi') of 32 spot pairs
  float2 B1 = make_float2(0.0f, 0.0f), B2 = B1, B3 = B1, B4 = B1;
  // y and exp(+i 2 pi base) of spots (n0 + 2 lane, n0 + 2 lane + 1) of
  // chunk j of group s
  auto fetch_y = [&](bool in, int s, int j, float4& yv, float4& rv) {
    yv = rv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (!in) return;
    const int tile = s / kTcGroupsPerTile;
    const int n = j * kTcChunk + 2 * lane;
    if (n < N) {
      const float2 a = __ldg(p.y + n), b = __ldg(p.rot + (size_t)tile * N + n);
      yv.x = a.x; yv.y = a.y; rv.x = b.x; rv.y = b.y;
    }
    if (n + 1 < N) {
      const float2 a = __ldg(p.y + n + 1), b = __ldg(p.rot + (size_t)tile * N + n + 1);
      yv.z = a.x; yv.w = a.y; rv.z = b.x; rv.w = b.y;
    }
  };
  float4 yv, rv;
  fetch_y(nc > 0, s0, j0, yv, rv);

  int s = s0, jch = j0;              // group and spot chunk of chunk c
  for (int c = 0; c < nc; ++c) {
    const bool last_of_group = jch + 1 == nch || c == nc - 1;
    const int s_next = jch + 1 == nch ? s + 1 : s, j_next = jch + 1 == nch ? 0 : jch + 1;
    const int valid = min(kTcChunk, N - jch * kTcChunk);
    const int nq = (valid + 15) >> 4;
    uint32_t x[4][16];
    ok = ok && mbar_wait(&full[c & 1], (uint32_t)((c >> 1) & 1), kTcWaitPolls);
    tc_fence_after();
    tc_load_cols(tmem + tlane + (uint32_t)((c & 1) * kTcChunk), 0, nq, x);
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      const uint32_t order = atom_add_acq_rel_smem(&cnt[c & 1], 1u) & 3u;
      if (order == 3u) {
        // every warp is done with TMEM buffer c & 1
        tc_fence_after();
        ok = issue_upto(c + 2) && ok;
      } else if (order == 0u) {
        // MMA(c) has completed (this warp saw it), and with it every MMA
        // of group s once c is the group's last chunk
        if (c + NB < nc) load_b(c + NB, jb);
        if (last_of_group && s + 2 <= s_last) load_a(s + 2);
      }
    }
    __syncwarp();
    if (++jb == nch) jb = 0;
    // y' = y exp(+i 2 pi base) of this chunk into the warp's slot
    yw[lane] = make_float4(yv.x * rv.x - yv.y * rv.y, yv.z * rv.z - yv.w * rv.w, yv.x * rv.y + yv.y * rv.x,
                           yv.z * rv.w + yv.w * rv.z);
    __syncwarp();
    fetch_y(c + 1 < nc, s_next, j_next, yv, rv);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q < nq) {
#pragma unroll
        for (int pp = 0; pp < 8; ++pp) {
          const float4 yq = yw[8 * q + pp];
          const float2 yr = make_float2(yq.x, yq.y), yi = make_float2(yq.z, yq.w);
          float2 sn, cs;
          // the local phase in turns
          sincos2_turns_mixed<ASH_POLY_ADJ, REDUCE>(
              8 * q + pp, make_float2(__uint_as_float(x[q][2 * pp]), __uint_as_float(x[q][2 * pp + 1])), sn, cs);
          // y exp(+i x) = (yr cs - yi sn) + i (yi cs + yr sn)
          B1 = fma2(yr, cs, B1);
          B2 = fma2(yi, sn, B2);
          B3 = fma2(yi, cs, B3);
          B4 = fma2(yr, sn, B4);
        }
      }
    }
    __syncwarp();   // the slot is rewritten for the next chunk
    if (last_of_group) {
      const float gr = (B1.x + B1.y) - (B2.x + B2.y), gi = (B3.x + B3.y) + (B4.x + B4.y);
      B1 = B2 = B3 = B4 = make_float2(0.0f, 0.0f);
      if ((long long)s * nch >= u0 && (long long)(s + 1) * nch <= u1) {
        tc_adjoint_epilogue(p, 2LL * s + (t >> 6), t & 63, gr, gi);
      } else {
        p.split[((size_t)cta * 2 + (s == s0 ? 0 : 1)) * kTcRows + t] = make_float2(gr, gi);
      }
    }
    s = s_next;
    jch = j_next;
  }
  tc_range_end(bars, armed, NBARS);
  if (!ok && t == 0) atomicOr(p.err, kErrTimeout);
}

// REDUCE = false: the dL/dphi pass of a gradient (epilogue kEpiGradPhase),
// run once per gradient rather than inside a loop, feeds the MUFU the local
// phase unreduced (see sin2_turns_mixed).
template <int NA, bool REDUCE = true>
__global__ void __launch_bounds__(kTcThreads, 4) k_tc_adjoint(const TcAdjParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = tc_smem_base(smem_raw);
  const uint32_t tmem = tc_tmem_alloc(reinterpret_cast<uint32_t*>(base + TcAdjShape<NA>::TSLOT));
  const int g = blockIdx.x;
  tc_adjoint_range<NA, REDUCE>(p, p.begin[g], p.begin[g + 1], g, base, tmem, true);
  tc_tmem_free(tmem);
}

// Batched form: CTA g of a launch over the concatenated units of many
// holograms (hologram h owns units [hu0[h], hu0[h + 1])) runs its slice of
// each hologram it meets, in order, as that hologram's local CTA g - g0[h].
template <int NA>
__global__ void __launch_bounds__(kTcThreads, 4) k_tc_adjoint_batch(const TcAdjParams* __restrict__ ps,
                                                                     const TcBatchSched bs) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = tc_smem_base(smem_raw);
  const uint32_t tmem = tc_tmem_alloc(reinterpret_cast<uint32_t*>(base + TcAdjShape<NA>::TSLOT));
  const int g = blockIdx.x;
  const long long B0 = bs.begin(g), B1 = bs.begin(g + 1);
  bool first = true;
  for (int h = bs.holo_of(B0); h < bs.count && bs.hu0[h] < B1; ++h) {
    const long long lu0 = max(B0, bs.hu0[h]) - bs.hu0[h], lu1 = min(B1, bs.hu0[h + 1]) - bs.hu0[h];
    if (lu1 <= lu0) continue;
    // this hologram's parameter block, staged in shared memory
    __shared__ TcAdjParams sp;
    __syncthreads();
    if (threadIdx.x == 0) sp = ps[h];
    __syncthreads();
    tc_adjoint_range<NA>(sp, lu0, lu1, g - bs.g0[h], base, tmem, first);
    first = false;
  }
  tc_tmem_free(tmem);
}

// Groups whose spots were split between CTAs of k_tc_adjoint: the partial
// sums in CTA order, then the epilogue. One CTA of 128 threads per split group.
// Group s, split over CTAs b_lo..b_hi (tabulated on the host).
__device__ __forceinline__ void tc_adjoint_fixup_group(const TcAdjParams& p, long long s, int b_lo, int b_hi) {
  const int nch = (p.g.N + kTcChunk - 1) / kTcChunk;
  const long long ulo = s * nch;
  const int t = threadIdx.x;
  float gr = 0.0f, gi = 0.0f;
  for (int cb = b_lo; cb <= b_hi; ++cb) {
    const long long beg = p.begin[cb];
    if (p.begin[cb + 1] <= beg) continue;
    const float2 v = p.split[((size_t)cb * 2 + (beg >= ulo ? 0 : 1)) * kTcRows + t];
    gr += v.x;
    gi += v.y;
  }
  tc_adjoint_epilogue(p, 2 * s + (t >> 6), t & 63, gr, gi);
}

static __global__ void k_tc_adjoint_fixup(const TcAdjParams p) {
  const int4 e = p.split_groups[blockIdx.x];
  tc_adjoint_fixup_group(p, e.x, e.y, e.z);
}

// Batched fix-up: entry i of `list` is (hologram, split group, first CTA, last CTA).
static __global__ void k_tc_adjoint_fixup_batch(const TcAdjParams* __restrict__ ps, const int4* __restrict__ list) {
  const int4 e = list[blockIdx.x];
  tc_adjoint_fixup_group(ps[e.x], e.y, e.z, e.w);
}

// --- forward ------------------------------------------------------------------

// E_n = sum_m f_m exp(-i C_n . Z_m) over this CTA's (spot block, pixel chunk)
// range; blocks whose pixels are split between CTAs go through `part` and
// k_tc_forward_reduce.
//
// Range of the forward's units this CTA runs, when the last spot block is
// replicated. Its chunks carry a quarter (or half) of a full chunk's
// arithmetic but the same MMAs, so two of its CTAs on one SM make that SM
// finish last; where the block scheduler puts a launch's CTAs depends on
// the kernels before it. Each SM's CTAs count themselves on a per-SM
// counter, and the last of them takes one of the replicated block's ranges
// (one per SM); the others take the full blocks' ranges in claim order. A CTA
// whose preferred pool is empty takes from the other, so every range is
// run exactly once whatever the placement (the results do not depend on
// which CTA runs a range: each writes its own partial sums).
__device__ __forceinline__ int tc_claim_range(int* claim, int n_full, int G, unsigned* err) {
  unsigned smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  const int slot = smid < (unsigned)kTcClaimSms ? atomicAdd(&claim[3 + smid], 1) : 0;
  const int n_rep = G - n_full;                 // one per SM
  const int per_sm = n_rep > 0 ? G / n_rep : 1;   // resident CTAs per SM
  const bool rep_first = slot % per_sm == per_sm - 1;
  for (int pass = 0; pass < 2; ++pass) {
    const bool rep = (pass == 0) == rep_first;
    const int k = atomicAdd(&claim[rep ? 1 : 0], 1);
    if (k < (rep ? n_rep : n_full)) return rep ? n_full + k : k;
  }
  atomicOr(err, kErrClaim);   // more CTAs than ranges: not launched that way
  return -1;
}

// The launch's last CTA zeroes the claim counters for the next launch
// (stream order makes them visible to it).
__device__ __forceinline__ void tc_claim_done(int* claim, int G) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&claim[2], 1) == G - 1;
  }
  __syncthreads();
  if (s_last) {
    for (int k = threadIdx.x; k < kTcClaimInts; k += blockDim.x) claim[k] = 0;
    __threadfence();
  }
}

// Producer schedule. The warp releasing chunk c last issues the MMAs up to
// chunk c + 2 (nothing else: the MMA is what the other warps wait for); the
// warp releasing it first loads B of chunk c + NBB into the slot MMA(c) has
// freed and f of chunk c + KF into the slot of chunk c + KF - NF = c - 3.
// No warp runs more than two chunks ahead of another (chunk c + 2's MMA
// needs every warp's release of c), so every warp has finished reading
// chunk c - 3's f. A spot block's first MMA waits until the previous
// block's last MMA has completed, then its A is reloaded (once per block
// change).
template <int NA>
__device__ __forceinline__ void tc_forward_range(const TcFwdParams& p, long long u0, long long u1, int cta,
                                                 uint8_t* base, uint32_t tmem, bool first_range) {
  using S = TcFwdShape<NA>;
  constexpr int NBB = S::NBB, KF = S::KF, NF = S::NF, NBARS = S::NBARS;
  float* sA = reinterpret_cast<float*>(base);                      // [NA][128][32]
  float* sB = sA + NA * 4096;                                      // [NBB][NA][64][32]
  float4* sF = reinterpret_cast<float4*>(sB + NBB * NA * 2048);    // [NF][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sF + NF * 32);      // full[2] | bfull[NBB] | ffull[NF] | afull
  uint64_t* full = bars;
  uint64_t* bfull = bars + 2;
  uint64_t* ffull = bars + 2 + NBB;
  uint64_t* afull = bars + 2 + NBB + NF;
  uint32_t* armed = reinterpret_cast<uint32_t*>(bars + NBARS);
  uint32_t* cnt = armed + NBARS;                                   // [2] arrivals per TMEM buffer
  uint32_t* tslot = cnt + 2;
  int* pst = reinterpret_cast<int*>(tslot + 1);   // next MMA: chunk, block, pixel chunk; block in A; A unchecked

  (void)tslot;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const Geometry& G = p.g;
  const int N = G.N;
  const int nq = G.T * kTcChunksPerTile;
  const int nc = (int)(u1 - u0);
  // chunk c of this range is pixel chunk q of spot block b; (b, q) advance
  // incrementally
  const int b0 = (int)(u0 / nq), q0 = (int)(u0 % nq);

  tc_range_begin(bars, armed, cnt, NBARS, first_range);
  const uint32_t tlane = (uint32_t)(w * 32) << 16;
  bool ok = true;

  // --- producer steps (one thread at a time) ---
  const int nb = p.sched.nb;
  // the last block uses its replicated image (chunks 2 nb, 2 nb + 1)
  auto load_a = [&](int b) {
    mbar_expect_tx(afull, S::A_BYTES);
    ++armed[NBARS - 1];
    const int chunk = (b == nb - 1 && p.rep > 1) ? 2 * nb : 2 * b;
    tc_copy_rows128<NA>(sA, p.czs + (size_t)chunk * NA * 2048, afull);
  };
  auto load_b = [&](int c, int q) {
    const int slot = c % NBB;
    mbar_expect_tx(&bfull[slot], S::B_BYTES);
    ++armed[2 + slot];
    bulk_g2s(sB + slot * NA * 2048, p.zs + (size_t)q * NA * 2048, S::B_BYTES, &bfull[slot]);
  };
  auto load_f = [&](int c, int q) {
    const int slot = c % NF;
    mbar_expect_tx(&ffull[slot], S::F_BYTES);
    ++armed[2 + NBB + slot];
    bulk_g2s(sF + slot * 32, p.fimg + (size_t)q * 32, S::F_BYTES, &ffull[slot]);
  };
  auto next_q = [&](int q) { return q + 1 == nq ? 0 : q + 1; };
  // MMAs of chunks pst[0] .. upto; `released`: the last chunk every warp has
  // released (its MMA and all earlier ones are complete)
  auto issue_upto = [&](int upto, int released) -> bool {
    bool r = true;
    int k = pst[0], b = pst[1], q = pst[2], ab = pst[3], fresh = pst[4];
    for (; k <= upto && k < nc;) {
      if (b != ab) {
        if (k - 1 > released) break;   // an MMA with the old block may still be running
        load_a(b);
        ab = b;
        fresh = 1;
      }
      r = mbar_wait(&bfull[k % NBB], (uint32_t)((k / NBB) & 1), kTcWaitPolls) && r;
      if (fresh) {
        r = mbar_wait(afull, (uint32_t)((b - b0) & 1), kTcWaitPolls) && r;
        fresh = 0;
      }
      tc_fence_after();
      ++armed[k & 1];
      tc_mma_chunk<NA>(tmem + (uint32_t)((k & 1) * kTcChunk), sA, sB + (k % NBB) * NA * 2048, &full[k & 1]);
      ++k;
      if (++q == nq) {
        q = 0;
        ++b;
      }
    }
    pst[0] = k;
    pst[1] = b;
    pst[2] = q;
    pst[3] = ab;
    pst[4] = fresh;
    return r;
  };

  int qb = q0, qf = q0;              // pixel chunks of chunks c + NBB and c + KF (the next to load)
  for (int k = 0; k < NBB; ++k) qb = next_q(qb);
  for (int k = 0; k < KF; ++k) qf = next_q(qf);
  if (t == 0 && nc > 0) {
    pst[0] = 0;
    pst[1] = b0;
    pst[2] = q0;
    pst[3] = b0;
    pst[4] = 1;
    load_a(b0);
    for (int c = 0, q = q0; c < NBB && c < nc; ++c, q = next_q(q)) load_b(c, q);
    for (int c = 0, q = q0; c < KF && c < nc; ++c, q = next_q(q)) load_f(c, q);
    ok = issue_upto(1, -1);
  }

  float2 A1 = make_float2(0.0f, 0.0f), A2 = A1;   // sums of A cos(phi - x), A sin(phi - x)
  float er = 0.0f, ei = 0.0f;
  int b = b0, q = q0;                // spot block and pixel chunk of chunk c
  // chunks [0, c_rep) belong to full blocks, [c_rep, nc) to the replicated
  // last block; the two passes are compiled separately
  const int c_rep = p.rep > 1 ? (int)min((long long)nc, max(0LL, (long long)(nb - 1) * nq - u0)) : nc;
  const bool had_rep = c_rep < nc;
  auto chunks = [&](auto tag, int c_beg, int c_end) {
    constexpr bool REPL = decltype(tag)::value;
    // replicated block: warp w takes columns [ri width, (ri + 1) width) for
    // the spots of rows t % spb
    const int spb = REPL ? kTcRows / p.rep : kTcRows;
    const int ri = REPL ? w / (4 / p.rep) : 0;
    const int width = REPL ? kTcChunk / p.rep : kTcChunk;
    const int g_lo = ri * width / 16, g_hi = g_lo + width / 16;
    for (int c = c_beg; c < c_end; ++c) {
      const bool wrap = q + 1 == nq;
      uint32_t x[4][16];
      ok = ok && mbar_wait(&full[c & 1], (uint32_t)((c >> 1) & 1), kTcWaitPolls);
      tc_fence_after();
      tc_load_cols(tmem + tlane + (uint32_t)((c & 1) * kTcChunk), REPL ? g_lo : 0, REPL ? g_hi : 4, x);
      tc_fence_before();
      __syncwarp();
      // a warp can be up to two chunks ahead of another (MMAs run two
      // chunks ahead), so arrivals are counted per TMEM buffer; the count
      // also tells the first and the last
      if (lane == 0) {
        const uint32_t order = atom_add_acq_rel_smem(&cnt[c & 1], 1u) & 3u;
        if (order == 3u) {
          // every warp is done with TMEM buffer c & 1
          tc_fence_after();
          ok = issue_upto(c + 2, c) && ok;
        } else if (order == 0u) {
          // MMA(c) has completed (this warp saw it) and every warp is done
          // with chunk c - 3
          if (c + NBB < nc) load_b(c + NBB, qb);
          if (c + KF < nc) load_f(c + KF, qf);
        }
      }
      __syncwarp();
      qb = next_q(qb);
      qf = next_q(qf);
      const int n = b * kTcRows + t % spb;
      // warps whose 32 spots are all >= N have nothing to add
      if (REPL || b * kTcRows + 32 * w < N) {
        ok = ok && mbar_wait(&ffull[c % NF], (uint32_t)((c / NF) & 1), kTcWaitPolls);
        const float4* f = sF + (c % NF) * 32;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          if (REPL && (qq < g_lo || qq >= g_hi)) continue;
#pragma unroll
          for (int pp = 0; pp < 8; ++pp) {
            const float4 fq = f[8 * qq + pp];
            const float2 am = make_float2(fq.x, fq.y), ph = make_float2(fq.z, fq.w);
            const float2 xv = make_float2(__uint_as_float(x[qq][2 * pp]), __uint_as_float(x[qq][2 * pp + 1]));
            float2 sn, cs;
            // f exp(-i x) = A exp(i 2 pi (phi - x)), phi and x in turns
            sincos2_turns_mixed<ASH_POLY_FWD>(8 * qq + pp, fma2(xv, make_float2(-1.0f, -1.0f), ph), sn, cs);
            A1 = fma2(am, cs, A1);
            A2 = fma2(am, sn, A2);
          }
        }
        if (q % kTcChunksPerTile == kTcChunksPerTile - 1 || c == nc - 1) {
          // end of a tile: rotate by exp(-i 2 pi base(n, tile))
          const float re = A1.x + A1.y, im = A2.x + A2.y;
          A1 = A2 = make_float2(0.0f, 0.0f);
          if (n < N) {
            const float2 rt = __ldg(p.rot + (size_t)(q / kTcChunksPerTile) * N + n);
            er += re * rt.x + im * rt.y;
            ei += im * rt.x - re * rt.y;
          }
        }
      }
      if (!REPL && (wrap || c == nc - 1)) {
        // end of spot block b in this range
        if ((long long)b * nq >= u0 && (long long)(b + 1) * nq <= u1) {
          if (n < N) p.E[n] = make_float2(er, ei);
        } else {
          p.part[((size_t)cta * 2 + (b == b0 ? 0 : 1)) * kTcRows + t] = make_float2(er, ei);
        }
        er = ei = 0.0f;
      }
      if (wrap) {
        q = 0;
        ++b;
      } else {
        ++q;
      }
    }
  };
  chunks(BoolTag<false>{}, 0, c_rep);
  if (had_rep) chunks(BoolTag<true>{}, c_rep, nc);
  tc_fence_before();
  __syncthreads();
  if (t == 0) tc_drain(bars, armed, NBARS);
  __syncwarp();
  if (had_rep) {
    // the replicated last block ends this range: sum the replicas in a fixed
    // order (every MMA has completed, so A's slot is free)
    __syncthreads();
    float2* red = reinterpret_cast<float2*>(sA);
    red[t] = make_float2(er, ei);
    __syncthreads();
    const int spb = kTcRows / p.rep;
    if (t < spb) {
      float sr = 0.0f, si = 0.0f;
      for (int k = 0; k < p.rep; ++k) {
        sr += red[t + k * spb].x;
        si += red[t + k * spb].y;
      }
      const int bl = nb - 1, n = bl * kTcRows + t;
      if ((long long)bl * nq >= u0 && (long long)(bl + 1) * nq <= u1) {
        if (n < N) p.E[n] = make_float2(sr, si);
      } else {
        p.part[((size_t)cta * 2 + (bl == b0 ? 0 : 1)) * kTcRows + t] = make_float2(sr, si);
      }
    }
  }
  tc_range_end(bars, armed, NBARS, /*drained=*/true);
  if (!ok && t == 0) atomicOr(p.err, kErrTimeout);
}

template <int NA>
__global__ void __launch_bounds__(kTcThreads, 4) k_tc_forward(const TcFwdParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = tc_smem_base(smem_raw);
  const uint32_t tmem = tc_tmem_alloc(reinterpret_cast<uint32_t*>(base + TcFwdShape<NA>::TSLOT));
  __shared__ int s_range;
  if (threadIdx.x == 0) s_range = p.claim ? tc_claim_range(p.claim, p.n_full, (int)gridDim.x, p.err) : blockIdx.x;
  __syncthreads();
  const int g = s_range;
  if (g >= 0) tc_forward_range<NA>(p, p.begin[g], p.begin[g + 1], g, base, tmem, true);
  if (p.claim) tc_claim_done(p.claim, (int)gridDim.x);
  tc_tmem_free(tmem);
}

// Batched form (see k_tc_adjoint_batch). Its parameter block comes from
// memory rather than the constant bank, which costs registers: three CTAs
// per SM instead of four.
template <int NA>
__global__ void __launch_bounds__(kTcThreads, 3) k_tc_forward_batch(const TcFwdParams* __restrict__ ps,
                                                                     const TcBatchSched bs) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = tc_smem_base(smem_raw);
  const uint32_t tmem = tc_tmem_alloc(reinterpret_cast<uint32_t*>(base + TcFwdShape<NA>::TSLOT));
  const int g = blockIdx.x;
  const long long B0 = bs.begin(g), B1 = bs.begin(g + 1);
  bool first = true;
  for (int h = bs.holo_of(B0); h < bs.count && bs.hu0[h] < B1; ++h) {
    const long long lu0 = max(B0, bs.hu0[h]) - bs.hu0[h], lu1 = min(B1, bs.hu0[h + 1]) - bs.hu0[h];
    if (lu1 <= lu0) continue;
    __shared__ TcFwdParams sp;
    __syncthreads();
    if (threadIdx.x == 0) sp = ps[h];
    __syncthreads();
    tc_forward_range<NA>(sp, lu0, lu1, g - bs.g0[h], base, tmem, first);
    first = false;
  }
  tc_tmem_free(tmem);
}

// Spot blocks whose pixels were split between CTAs of k_tc_forward: E_n is
// the sum of the CTAs' partial sums. CTA (b, y) sums 32 spots of block b:
// row-lane k of the 32 x 32 threads adds the partials of CTAs g_lo + k,
// g_lo + k + 32, ..., then a fixed-shape tree combines the row-lanes.
__device__ __forceinline__ void tc_forward_reduce_block(const TcFwdParams& p, long long b, int col, int g_lo,
                                                        int g_hi) {
  __shared__ float2 acc[32][33];
  const int nq = p.g.T * kTcChunksPerTile;
  const long long ulo = b * nq;
  const int k = threadIdx.y;
  if (g_lo == g_hi) return;   // one CTA owned the block and wrote E itself
  float2 v = make_float2(0.0f, 0.0f);
  for (int cb = g_lo + k; cb <= g_hi; cb += 32) {
    const long long beg = p.begin[cb];
    if (p.begin[cb + 1] <= beg) continue;
    const float2 x = p.part[((size_t)cb * 2 + (beg >= ulo ? 0 : 1)) * kTcRows + col];
    v.x += x.x;
    v.y += x.y;
  }
  acc[k][threadIdx.x] = v;
  __syncthreads();
  for (int h = 16; h > 0; h >>= 1) {
    if (k < h) {
      acc[k][threadIdx.x].x += acc[k + h][threadIdx.x].x;
      acc[k][threadIdx.x].y += acc[k + h][threadIdx.x].y;
    }
    __syncthreads();
  }
  const int n = (int)(b * kTcRows) + col;
  if (k == 0 && n < p.g.N) p.E[n] = acc[0][threadIdx.x];
}

static __global__ void k_tc_forward_reduce(const TcFwdParams p) {
  const int2 sp = p.spans[blockIdx.x];
  tc_forward_reduce_block(p, blockIdx.x, blockIdx.y * 32 + threadIdx.x, sp.x, sp.y);
}

// Batched reduction: entry i of `list` is (hologram, spot block, first CTA, last CTA).
static __global__ void k_tc_forward_reduce_batch(const TcFwdParams* __restrict__ ps, const int4* __restrict__ list) {
  const int4 e = list[blockIdx.x];
  tc_forward_reduce_block(ps[e.x], e.y, blockIdx.y * 32 + threadIdx.x, e.z, e.w);
}

// Nearfield images of a batch (one thread per pixel of the concatenated tiles).
static __global__ void k_tc_field_img_batch(const TcFieldDesc* __restrict__ ds, const int* __restrict__ tiles0,
                                            int count, int total_tiles) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)total_tiles * kTilePix) return;
  const int gt = (int)(e / kTilePix);
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (tiles0[mid] <= gt) lo = mid;
    else hi = mid - 1;
  }
  const TcFieldDesc& d = ds[lo];
  const long long le = e - (long long)tiles0[lo] * kTilePix;
  const long long qc = le / kTcChunk;
  const int r = (int)(le % kTcChunk);
  const Geometry& G = d.g;
  const TcPixel px = tc_pixel(G, qc, r);
  float a = 0.0f, ph = 0.0f;
  if (px.i < G.nx && px.j < G.ny) {
    a = d.amp_img[px.img];
    ph = turns_of_phase(d.phase[(size_t)px.j * G.nx + px.i]);
  }
  float* q = reinterpret_cast<float*>(d.fimg) + ((size_t)qc * 32 + (r >> 1)) * 4;
  q[r & 1] = a;
  q[2 + (r & 1)] = ph;
}

}  // namespace ash
