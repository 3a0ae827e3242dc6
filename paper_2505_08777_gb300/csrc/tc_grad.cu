// Coefficient gradient on the tensor cores: the spot-stationary moment pass
// dL/dC_nd = Im(conj(dL/dE_n) sum_m Z_dm f_m exp(-i C_n . Z_m)) (paper
// Methods, gradients of the spot field), with the phases C_n . dZ_m from the
// same split-tf32 MMA as the forward transform.
#include "tc_kernels.cuh"

namespace ash {

namespace {

// --- coefficient-gradient moments -----------------------------------------------

// Tile polynomials of the basis: over a 32 x 32 tile, x = x_c + s u and
// y = y_c + s v with u = (col - 15.5) / 16, v = (row - 15.5) / 16 and
// s = 16 / R, so a basis polynomial sum coef x^a y^b is
// sum_{k + l <= ORD} b_kl u^k v^l with
// b_kl = sum coef binom(a, k) x_c^(a-k) s^k binom(b, l) y_c^(b-l) s^l,
// exact in fp64 and rounded once. One thread per (tile, (k, l), mode);
// tpoly[tile][pair][DP], pairs in the order k = 0..ORD, l = 0..ORD-k; modes
// D..DP-1 are 0.
__global__ void k_tc_tile_poly(const Geometry G, const MonoTerm* __restrict__ terms, const int* __restrict__ term_off,
                               int ord, int DP, float* __restrict__ tpoly) {
  const int npair = (ord + 1) * (ord + 2) / 2;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)G.T * npair * DP) return;
  const int d = (int)(e % DP);
  const int pr = (int)((e / DP) % npair);
  const int tile = (int)(e / ((long long)DP * npair));
  int k = 0, l = pr;
  while (l > ord - k) {
    l -= ord - k + 1;
    ++k;
  }
  const double xc = grid_x(G, (double)((tile % G.tiles_x) * kTileX) + 15.5);
  const double yc = grid_y(G, (double)((tile / G.tiles_x) * kTileY) + 15.5);
  const double sc = 16.0 / grid_radius(G);
  double acc = 0.0;
  if (d < G.D) {
    for (int t = term_off[d]; t < term_off[d + 1]; ++t) {
      const MonoTerm m = terms[t];
      if (k > m.px || l > m.py) continue;
      // binom(a, k) x_c^(a-k) s^k and binom(b, l) y_c^(b-l) s^l
      double fx = 1.0, fy = 1.0;
      for (int r = 0; r < k; ++r) fx = fx * (double)(m.px - r) / (double)(r + 1) * sc;
      for (int r = 0; r < m.px - k; ++r) fx *= xc;
      for (int r = 0; r < l; ++r) fy = fy * (double)(m.py - r) / (double)(r + 1) * sc;
      for (int r = 0; r < m.py - l; ++r) fy *= yc;
      acc += m.coef * fx * fy;
    }
  }
  tpoly[((size_t)tile * npair + pr) * DP + d] = (float)acc;
}

// Shared memory of the moment kernel: A (spot block), B ring and f ring.
struct TcGradShape {
  static constexpr int NBB = 4, KF = 5, NF = KF + 3;   // as the forward's rings
  static constexpr uint32_t A_BYTES = 16384, B_BYTES = 8192, F_BYTES = 512;
  static constexpr uint32_t FSLOT = F_BYTES;
  static constexpr int NBARS = 3 + NBB + NF;
  static constexpr size_t SMEM = 1024 + A_BYTES + NBB * B_BYTES + NF * FSLOT + NBARS * 12 + 8 + 32;
};

// S_nd = sum_m Z_dm f_m exp(-i C_n . Z_m) and dL/dC_nd = Im(conj(gE_n) S_nd)
// (paper Methods, gradients through the kernels). With C_n . Z_m = 2 pi base
// + x (x the local phase from the tensor core) and w = conj(gE_n exp(+i 2 pi
// base)) = |w| exp(i alpha), constant over a tile, each term adds q Z_dm
// with q = Im(w f_m exp(-i x)) = |w| A_m sin(phi_m + alpha - x) (the
// nearfield image holds f = A exp(i phi) as (A, phi / 2 pi), the tensor
// core gives x / 2 pi, and the sine is taken of the sum in turns); |w| is
// applied once per tile. Over a tile Z_dm = sum_{k + l <= ORD} b_dkl u^k v^l (u, v the
// pixel's column and row offsets), so thread t (spot t of the block)
// accumulates along each row the power moments P_k = sum q u^k (u^k
// compile-time constants here), folds them into the tile moments
// Q_kl += v^l P_k at the row's end, and adds sum_kl b_dkl Q_kl to its D
// gradients at the tile's end.
template <int ORD, int DP>
__global__ void __launch_bounds__(kTcThreads, 4) k_tc_gradc(const TcGradParams p) {
  using S = TcGradShape;
  constexpr int NPOW = ORD + 1, NPAIR = (ORD + 1) * (ORD + 2) / 2;
  constexpr int NA = 1, NBB = S::NBB, KF = S::KF, NF = S::NF, NBARS = S::NBARS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = tc_smem_base(smem_raw);
  float* sA = reinterpret_cast<float*>(base);
  float* sB = sA + 4096;
  uint8_t* sFZ = reinterpret_cast<uint8_t*>(sB + NBB * 2048);     // [NF][f | dz pairs]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sFZ + NF * S::FSLOT);
  uint64_t* full = bars;
  uint64_t* bfull = bars + 2;
  uint64_t* ffull = bars + 2 + NBB;
  uint64_t* afull = bars + 2 + NBB + NF;
  uint32_t* armed = reinterpret_cast<uint32_t*>(bars + NBARS);
  uint32_t* cnt = armed + NBARS;
  uint32_t* tslot = cnt + 2;
  int* pst = reinterpret_cast<int*>(tslot + 1);
  const uint32_t tmem = tc_tmem_alloc(tslot);

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const Geometry& G = p.g;
  const int N = G.N, D = G.D;
  const int nq = G.T * kTcChunksPerTile;
  const long long u0 = p.begin[blockIdx.x], u1 = p.begin[blockIdx.x + 1];
  const int nc = (int)(u1 - u0);
  const int b0 = (int)(u0 / nq), q0 = (int)(u0 % nq);
  tc_range_begin(bars, armed, cnt, NBARS, true);
  const uint32_t tlane = (uint32_t)(w * 32) << 16;
  bool ok = true;

  auto load_a = [&](int b) {
    mbar_expect_tx(afull, S::A_BYTES);
    ++armed[NBARS - 1];
    tc_copy_rows128<NA>(sA, p.czs + (size_t)(2 * b) * 2048, afull);
  };
  auto load_b = [&](int c, int q) {
    const int slot = c % NBB;
    mbar_expect_tx(&bfull[slot], S::B_BYTES);
    ++armed[2 + slot];
    bulk_g2s(sB + slot * 2048, p.zs + (size_t)q * 2048, S::B_BYTES, &bfull[slot]);
  };
  auto load_f = [&](int c, int q) {
    const int slot = c % NF;
    uint8_t* dst = sFZ + slot * S::FSLOT;
    mbar_expect_tx(&ffull[slot], S::F_BYTES);
    ++armed[2 + NBB + slot];
    bulk_g2s(dst, p.fimg + (size_t)q * 32, S::F_BYTES, &ffull[slot]);
  };
  auto next_q = [&](int q) { return q + 1 == nq ? 0 : q + 1; };
  auto issue_upto = [&](int upto, int released) -> bool {
    bool r = true;
    int k = pst[0], b = pst[1], q = pst[2], ab = pst[3], fresh = pst[4];
    for (; k <= upto && k < nc;) {
      if (b != ab) {
        if (k - 1 > released) break;
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
      tc_mma_chunk<NA>(tmem + (uint32_t)((k & 1) * kTcChunk), sA, sB + (k % NBB) * 2048, &full[k & 1]);
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

  int qb = q0, qf = q0;
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

  float dc[DP], Q[NPAIR];
#pragma unroll
  for (int d = 0; d < DP; ++d) dc[d] = 0.0f;
#pragma unroll
  for (int k = 0; k < NPAIR; ++k) Q[k] = 0.0f;
  float2 gh = make_float2(0.0f, 0.0f), alpha2 = gh;
  float wmag = 0.0f;
  int b = b0, q = q0;

  for (int c = 0; c < nc; ++c) {
    const bool wrap = q + 1 == nq;
    const int n = b * kTcRows + t;
    const bool active = b * kTcRows + 32 * w < N;
    if (c == 0 || q == 0) gh = n < N ? __ldg(p.gE + n) : make_float2(0.0f, 0.0f);   // new spot block
    if (c == 0 || q % kTcChunksPerTile == 0) {
      // new tile: w = conj(gE exp(+i 2 pi base(n, tile)))
      const float2 rt = n < N ? __ldg(p.rot + (size_t)(q / kTcChunksPerTile) * N + n) : make_float2(0.0f, 0.0f);
      // w = |w| exp(i alpha): q = Im(w f exp(-i x)) = |w| Im(f exp(-i (x - alpha)))
      const float wr = gh.x * rt.x - gh.y * rt.y, wi = -(gh.x * rt.y + gh.y * rt.x);
      const float alpha = atan2f(wi, wr) * 0.15915494309189535f;   // turns, as phi and x
      alpha2 = make_float2(alpha, alpha);
      wmag = sqrtf(wr * wr + wi * wi);
    }
    // row 0 of the chunk is TMEM columns 0-31, row 1 columns 32-63; the
    // buffer is released once both are in registers
    const uint32_t taddr = tmem + tlane + (uint32_t)((c & 1) * kTcChunk);
    const float4* f = reinterpret_cast<const float4*>(sFZ + (c % NF) * S::FSLOT);
    // rows 4h + 2 half and 4h + 2 half + 1 of the tile (chunk w = 2h + half)
    const int wq = q % kTcChunksPerTile;
    const float vr0 = ((float)(4 * (wq >> 1) + 2 * (wq & 1)) - 15.5f) * 0.0625f;
    auto row = [&](const uint32_t (&x)[2][16], int hr) {
      float P[NPOW];
#pragma unroll
      for (int k = 0; k < NPOW; ++k) P[k] = 0.0f;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 fq = f[16 * hr + k];
        const float2 am = make_float2(fq.x, fq.y), ph = make_float2(fq.z, fq.w);
        const float2 xv =
            make_float2(__uint_as_float(x[k / 8][2 * (k % 8)]), __uint_as_float(x[k / 8][2 * (k % 8) + 1]));
        // q / |w| = Im(A exp(i phi) exp(-i (x - alpha))) = A sin(phi + alpha - x)
        float2 sn;
        // the sine's argument goes to the MUFU unreduced: this pass runs
        // once per gradient, not inside a loop, and its error stays far
        // below the gradient's tolerance (c4, 32 spots: 1.3e-6 normwise
        // against 8.0e-7 reduced), for 12 % less time (647 -> 569 us)
        sin2_turns_mixed<ASH_POLY_GRAD, false>(
            16 * hr + k, fma2(xv, make_float2(-1.0f, -1.0f), fma2(ph, make_float2(1.0f, 1.0f), alpha2)), sn);
        const float2 qv = mul2(am, sn);
        // columns 2k, 2k + 1 of the row
        const float u0 = (2.0f * k - 15.5f) * 0.0625f, u1 = (2.0f * k + 1.0f - 15.5f) * 0.0625f;
        float p0 = 1.0f, p1 = 1.0f;
#pragma unroll
        for (int e = 0; e < NPOW; ++e) {
          P[e] = fmaf(qv.x, p0, P[e]);
          P[e] = fmaf(qv.y, p1, P[e]);
          p0 *= u0;
          p1 *= u1;
        }
      }
      // Q_kl += v^l P_k (v the row's offset)
      const float v = vr0 + 0.0625f * (float)hr;
      float vp[NPOW];
      vp[0] = 1.0f;
#pragma unroll
      for (int e = 1; e < NPOW; ++e) vp[e] = vp[e - 1] * v;
      int idx = 0;
#pragma unroll
      for (int e = 0; e < NPOW; ++e) {
#pragma unroll
        for (int l = 0; l + e < NPOW; ++l) {
          Q[idx] = fmaf(vp[l], P[e], Q[idx]);
          ++idx;
        }
      }
    };
    uint32_t x[2][16];
    ok = ok && mbar_wait(&full[c & 1], (uint32_t)((c >> 1) & 1), kTcWaitPolls);
    tc_fence_after();
    tmem_ld16_nowait(taddr, x[0]);
    tmem_ld16_nowait(taddr + 16, x[1]);
    tmem_wait();
    if (active) {
      ok = ok && mbar_wait(&ffull[c % NF], (uint32_t)((c / NF) & 1), kTcWaitPolls);
      row(x, 0);
    }
    tmem_ld16_nowait(taddr + 32, x[0]);
    tmem_ld16_nowait(taddr + 48, x[1]);
    tmem_wait();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      // the forward's producer schedule: the last warp to release chunk c
      // issues the MMAs up to c + 2, the first loads B of c + NBB and f of
      // c + KF (into chunk c - 3's slot)
      const uint32_t order = atom_add_acq_rel_smem(&cnt[c & 1], 1u) & 3u;
      if (order == 3u) {
        tc_fence_after();
        ok = issue_upto(c + 2, c) && ok;
      } else if (order == 0u) {
        if (c + NBB < nc) load_b(c + NBB, qb);
        if (c + KF < nc) load_f(c + KF, qf);
      }
    }
    __syncwarp();
    qb = next_q(qb);
    qf = next_q(qf);
    if (active) row(x, 1);
    if (active && (q % kTcChunksPerTile == kTcChunksPerTile - 1 || c == nc - 1)) {
      // end of a tile (or of the range): dC_d += |w| sum_kl b_dkl Q_kl
#pragma unroll
      for (int k = 0; k < NPAIR; ++k) Q[k] *= wmag;
      const float4* tb = reinterpret_cast<const float4*>(p.tpoly + (size_t)(q / kTcChunksPerTile) * NPAIR * DP);
#pragma unroll
      for (int k = 0; k < NPAIR; ++k) {
#pragma unroll
        for (int j = 0; j < DP / 4; ++j) {
          const float4 bv = __ldg(tb + k * (DP / 4) + j);
          dc[4 * j] = fmaf(bv.x, Q[k], dc[4 * j]);
          dc[4 * j + 1] = fmaf(bv.y, Q[k], dc[4 * j + 1]);
          dc[4 * j + 2] = fmaf(bv.z, Q[k], dc[4 * j + 2]);
          dc[4 * j + 3] = fmaf(bv.w, Q[k], dc[4 * j + 3]);
        }
        Q[k] = 0.0f;
      }
    }
    if (wrap || c == nc - 1) {
      // end of spot block b in this range
      const bool whole = (long long)b * nq >= u0 && (long long)(b + 1) * nq <= u1;
#pragma unroll
      for (int d = 0; d < DP; ++d) {
        if (whole) {
          if (n < N && d < D) p.dC[(size_t)n * D + d] = dc[d];
        } else {
          p.part[(((size_t)blockIdx.x * 2 + (b == b0 ? 0 : 1)) * kTcRows + t) * DP + d] = dc[d];
        }
        dc[d] = 0.0f;
      }
    }
    if (wrap) {
      q = 0;
      ++b;
    } else {
      ++q;
    }
  }
  tc_range_end(bars, armed, NBARS);
  if (!ok && t == 0) atomicOr(p.err, kErrTimeout);
  tc_tmem_free(tmem);
}

// Spot blocks of k_tc_gradc split between CTAs: dC_nd is the sum of the
// partial sums. CTA (b, spot group of 32, mode d): as k_tc_forward_reduce.
__global__ void k_tc_gradc_reduce(const TcGradParams p) {
  __shared__ float acc[32][33];
  const int nq = p.g.T * kTcChunksPerTile, DP = tc_grad_dp(p.g.D);
  const long long b = blockIdx.x, ulo = b * nq;
  const int col = blockIdx.y * 32 + threadIdx.x, d = blockIdx.z, k = threadIdx.y;
  const int g_lo = p.spans[b].x, g_hi = p.spans[b].y;
  if (g_lo == g_hi) return;
  float v = 0.0f;
  for (int cb = g_lo + k; cb <= g_hi; cb += 32) {
    const long long beg = p.begin[cb];
    if (p.begin[cb + 1] <= beg) continue;
    v += p.part[(((size_t)cb * 2 + (beg >= ulo ? 0 : 1)) * kTcRows + col) * DP + d];
  }
  acc[k][threadIdx.x] = v;
  __syncthreads();
  for (int h = 16; h > 0; h >>= 1) {
    if (k < h) acc[k][threadIdx.x] += acc[k + h][threadIdx.x];
    __syncthreads();
  }
  const int n = (int)(b * kTcRows) + col;
  if (k == 0 && n < p.g.N) p.dC[(size_t)n * p.g.D + d] = acc[0][threadIdx.x];
}

}  // namespace

template <int ORD, int DP>
static cudaError_t launch_np(const TcGradParams& p, cudaStream_t s) {
  k_tc_gradc<ORD, DP><<<p.sched.G, kTcThreads, TcGradShape::SMEM, s>>>(p);
  return cudaGetLastError();
}

template <int ORD, int DP>
static cudaError_t prepare_np(int* n) {
  const void* k = (const void*)k_tc_gradc<ORD, DP>;
  constexpr int smem = (int)TcGradShape::SMEM;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared)))
    return e;
  return tc_ctas_per_sm(k, smem, 2 * kTcChunk, n);
}

// Instantiations: ORD in 1..4, DP in {4, 8, 12}.
template <int ORD>
static cudaError_t dispatch_dp(int DP, bool prep, const TcGradParams* p, int* n, cudaStream_t s) {
  switch (DP) {
    case 4: return prep ? prepare_np<ORD, 4>(n) : launch_np<ORD, 4>(*p, s);
    case 8: return prep ? prepare_np<ORD, 8>(n) : launch_np<ORD, 8>(*p, s);
    case 12: return prep ? prepare_np<ORD, 12>(n) : launch_np<ORD, 12>(*p, s);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t dispatch(int ord, int DP, bool prep, const TcGradParams* p, int* n, cudaStream_t s) {
  switch (ord) {
    case 1: return dispatch_dp<1>(DP, prep, p, n, s);
    case 2: return dispatch_dp<2>(DP, prep, p, n, s);
    case 3: return dispatch_dp<3>(DP, prep, p, n, s);
    case 4: return dispatch_dp<4>(DP, prep, p, n, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tc_grad_prepare(int ord, int D, int* ctas_per_sm) {
  return dispatch(ord, tc_grad_dp(D), true, nullptr, ctas_per_sm, nullptr);
}

cudaError_t tc_build_tile_poly(const Geometry& g, const MonoTerm* terms, const int* term_off, int ord, float* tpoly,
                               cudaStream_t s) {
  const int DP = tc_grad_dp(g.D);
  const long long n = (long long)g.T * tc_grad_pairs(ord) * DP;
  k_tc_tile_poly<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, terms, term_off, ord, DP, tpoly);
  return cudaGetLastError();
}

cudaError_t tc_launch_gradc(const TcGradParams& p, bool split, cudaStream_t s) {
  cudaError_t e = dispatch(p.ord, tc_grad_dp(p.g.D), false, &p, nullptr, s);
  if (e != cudaSuccess || !split) return e;
  k_tc_gradc_reduce<<<dim3(p.sched.nb, kTcRows / 32, p.g.D), dim3(32, 32), 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace ash
