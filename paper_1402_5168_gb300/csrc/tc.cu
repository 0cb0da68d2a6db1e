// Leaf down-solves on the tensor cores (tcgen05, bf16 slices, FP32 accumulation in
// TMEM), with the pole sum fused into the epilogue.
//
// The leaf down-solve of pole p (Section 2.3: interior values from the leaf's
// solution operators) is x_p = X_p g_p + Y_p u_b with g_p = sum_k c_pk s_k, s_k the
// pre-mapped sources of the state (pole independent) and u_b the leaf's edge values
// of pole p.  The coefficients are folded into the operator once, at build time:
//     x_p = A'_p [s_0; ...; s_{K-1}; u_b],   A'_p = [c_p0 X_p | ... | c_p,K-1 X_p | Y_p],
// so the K source blocks are pole independent and split into bf16 slices once per
// step, and only u_b is split per pole.  Each real part of A' and of the right-hand
// sides is split into S slices (tc.cuh) with a power-of-two scale per operator row
// and per right-hand-side column, separately for the source and the edge blocks.
// The products of the slices run as tcgen05.mma (M = 128 operator rows, N = 32
// right-hand-side columns, K = 16), accumulated in TMEM in three levels per block
// and component: i + j = 2 and i + j = 3 exactly, i + j = 4 .. S + 1 rounded.  The
// epilogue rescales and sums the levels in FP32 pairs (hi, lo), then adds
// Re(w_pk x_p) for every accumulation weight k into per-thread FP32-pair sums; the
// pole chunk's sums go to the same partial-sum array the other leaf kernels fill.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sweep.cuh"
#include "tc.cuh"

namespace eo {

// ---------------------------------------------------------------- build: operator split
// One block per (pole of the group, operator box, M tile); thread t owns row
// mt * 128 + t.  A' columns: kappa = kk * ni + j (kk < K, j < ni): c_p,kk X[row][j];
// then the edge block j' < nb: Y[row][j'] = XY[row][ni + j'].  Output per
// (pole, box, M tile, K step): 2S slice blocks (re slices, then im slices), and per
// row the two split exponents (source block, edge block).
template <int S>
__global__ void __launch_bounds__(128) k_tc_split_operator(int ni, int nb, int K, int nks, int nke, int nbox_op,
                                                            int pg0, const cd* __restrict__ XY, long long xps,
                                                            long long xbs, const cd* __restrict__ coef,
                                                            __nv_bfloat16* __restrict__ Aop, int* __restrict__ Aexp) {
  const int mt = blockIdx.x % 2, box = (blockIdx.x / 2) % nbox_op, gi = blockIdx.x / (2 * nbox_op);
  const int p = pg0 + gi;
  const int row = mt * tc::MT + threadIdx.x;
  const bool ok = row < ni;
  const cd* A = XY + (long long)gi * xps + (long long)box * xbs;
  const int kx = ni + nb;
  cd cf[3];
  for (int kk = 0; kk < K; ++kk) cf[kk] = coef[p * K + kk];
  // split exponents of the row's source block and edge block
  double ms = 0.0, me = 0.0;
  if (ok) {
    for (int kk = 0; kk < K; ++kk)
      for (int j = 0; j < ni; ++j) {
        const cd x = A[row + (size_t)j * ni];
        const double re = cf[kk].x * x.x - cf[kk].y * x.y, im = cf[kk].x * x.y + cf[kk].y * x.x;
        ms = fmax(ms, fmax(fabs(re), fabs(im)));
      }
    for (int j = 0; j < nb; ++j) {
      const cd x = A[row + (size_t)(ni + j) * ni];
      me = fmax(me, fmax(fabs(x.x), fabs(x.y)));
    }
  }
  const int es = tc::split_exponent(ms), ee = tc::split_exponent(me);
  const size_t opi = ((size_t)p * nbox_op + box) * 2 + mt;
  Aexp[opi * 2 * tc::MT + threadIdx.x] = es;
  Aexp[opi * 2 * tc::MT + tc::MT + threadIdx.x] = ee;
  const int nk = nks + nke;
  __nv_bfloat16* out = Aop + opi * (size_t)nk * 2 * S * (tc::A_BLK / 2);
  float sr[S], si[S];
  for (int ks = 0; ks < nk; ++ks) {
    __nv_bfloat16* blk = out + (size_t)ks * 2 * S * (tc::A_BLK / 2);
    for (int k = 0; k < tc::KS; ++k) {
      double re = 0.0, im = 0.0;
      int e = es;
      if (ok) {
        if (ks < nks) {
          const int kap = ks * tc::KS + k;
          if (kap < K * ni) {
            const int kk = kap / ni, j = kap - kk * ni;
            const cd x = A[row + (size_t)j * ni];
            re = cf[kk].x * x.x - cf[kk].y * x.y;
            im = cf[kk].x * x.y + cf[kk].y * x.x;
          }
        } else {
          const int j = (ks - nks) * tc::KS + k;
          e = ee;
          if (j < nb) {
            const cd x = A[row + (size_t)(ni + j) * ni];
            re = x.x;
            im = x.y;
          }
        }
      }
      tc::split_value<S>(re, e, sr);
      tc::split_value<S>(im, e, si);
      const int o = tc::core_off(threadIdx.x, k);
#pragma unroll
      for (int i = 0; i < S; ++i) {
        blk[(size_t)i * (tc::A_BLK / 2) + o] = __float2bfloat16_rn(sr[i]);
        blk[(size_t)(S + i) * (tc::A_BLK / 2) + o] = __float2bfloat16_rn(si[i]);
      }
    }
  }
  (void)kx;
}

// Column of right-hand-side tile t, slot n: (box, rhs), or box = -1 past the end.
// Per-box operators: a tile holds right-hand sides of one box; shared operators: any.
__device__ __forceinline__ void tc_column(int shared, int R, int nleaf, int t, int n, int& box, int& r) {
  if (shared) {
    const int col = t * tc::NT + n;
    box = col / R;
    r = col - box * R;
    if (box >= nleaf) box = -1;
  } else {
    const int tpb = (R + tc::NT - 1) / tc::NT;
    box = t / tpb;
    r = (t - box * tpb) * tc::NT + n;
    if (r >= R) box = -1;
  }
}

// ---------------------------------------------------------------- per step: source split
// One block per right-hand-side tile: the pole-independent source block of every
// column (kappa = kk * ni + j: s_kk at interior node j of the column's leaf), split
// relative to the column's exponent into S slices in the tile layout of the MMA.
template <int S>
__global__ void __launch_bounds__(256) k_tc_split_sources(Sweep s, int nleaf, int nks, __nv_bfloat16* __restrict__ Bs,
                                                           int* __restrict__ Bexp) {
  __shared__ int ecol[tc::NT];
  const int t = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ni = s.ni, nsrc = s.K * ni;
  // column exponents: warp w takes columns 4w .. 4w + 3
  for (int n = warp * 4; n < warp * 4 + 4; ++n) {
    int box, r;
    tc_column(s.shared, s.R, nleaf, t, n, box, r);
    double m = 0.0;
    if (box >= 0)
      for (int kap = lane; kap < nsrc; kap += 32) {
        const int kk = kap / ni, j = kap - kk * ni;
        m = fmax(m, fabs(s.src[kk][r * s.src_rs[kk] + (long long)box * ni + j]));
      }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) ecol[n] = tc::split_exponent(m);
  }
  __syncthreads();
  if (threadIdx.x < tc::NT) Bexp[t * tc::NT + threadIdx.x] = ecol[threadIdx.x];
  __nv_bfloat16* out = Bs + (size_t)t * nks * S * (tc::B_BLK / 2);
  float sl[S];
  for (int e = threadIdx.x; e < nks * tc::KS * tc::NT; e += blockDim.x) {
    const int n = e % tc::NT, kap = e / tc::NT, ks = kap / tc::KS, k = kap % tc::KS;
    int box, r;
    tc_column(s.shared, s.R, nleaf, t, n, box, r);
    double v = 0.0;
    if (box >= 0 && kap < nsrc) {
      const int kk = kap / ni, j = kap - kk * ni;
      v = s.src[kk][r * s.src_rs[kk] + (long long)box * ni + j];
    }
    tc::split_value<S>(v, ecol[n], sl);
    __nv_bfloat16* blk = out + (size_t)ks * S * (tc::B_BLK / 2);
    const int o = tc::core_off(n, k);
#pragma unroll
    for (int i = 0; i < S; ++i) blk[(size_t)i * (tc::B_BLK / 2) + o] = __float2bfloat16_rn(sl[i]);
  }
}

// ---------------------------------------------------------------- FP32 pairs (hi, lo)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  h = __fadd_rn(p, e);
  l = __fsub_rn(e, __fsub_rn(h, p));
}
// three FP32 levels (the first two exact) summed into a pair, times 2^e
__device__ __forceinline__ void levels(float a2, float a3, float a4, int e, float& h, float& l) {
  two_sum(a2, a3, h, l);
  df_add(h, l, a4, 0.0f);
  h = ldexpf(h, e);
  l = ldexpf(l, e);
}

struct TcArgs {
  Sweep s;
  int nleaf, nks, nke, nbox_op, ppc;
  const __nv_bfloat16* Aop;   // [P][nbox_op][2 M tiles][nk][2S][MT x KS]
  const int* Aexp;            // [P][nbox_op][2 M tiles][2][MT]
  const __nv_bfloat16* Bs;    // [tiles][nks][S][NT x KS]
  const int* Bexp;            // [tiles][NT]
  const cd* E;                // [pole in call][R][n_edge]
  const int* bseg;            // [nleaf][4]
  double* part;               // [chunk][R][K][n_int]
  int* status;                // set to 1 when a bounded wait gives up
};

constexpr int TC_STAGES = 4;
constexpr int TC_AHEAD = 2;          // bulk copies issued this many K steps ahead
constexpr long long TC_SPIN = 1LL << 20;

template <int S>
__host__ __device__ constexpr int tc_stage_bytes() { return 2 * S * (tc::A_BLK + tc::B_BLK); }

// Grid (right-hand-side tiles, 2 M tiles, pole chunks), 256 threads, one block per SM
// (TMEM: 12 accumulators of NT columns; shared memory: TC_STAGES stages).
template <int S>
__global__ void __launch_bounds__(256, 1) k_tc_down_leaf(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ __align__(8) uint64_t mb_tma[TC_STAGES], mb_mma[TC_STAGES];
  __shared__ uint32_t tmem_slot;
  __shared__ int eS[tc::NT], eE[tc::NT], boxof[tc::NT], rof[tc::NT];
  __shared__ float wdf[3][4];
  __shared__ int s_abort;
  const Sweep& s = a.s;
  const int t = blockIdx.x, mt = blockIdx.y, chunk = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = a.nks + a.nke, ni = s.ni, nb = s.nb, q = s.q, K = s.K;
  constexpr int SB = tc_stage_bytes<S>();
  const int pbeg = chunk * a.ppc, pend = min(s.P, pbeg + a.ppc);
  const int npole = max(0, pend - pbeg);
  const int total = npole * nk;
  if (tid < tc::NT) {
    int box, r;
    tc_column(s.shared, s.R, a.nleaf, t, tid, box, r);
    boxof[tid] = box;
    rof[tid] = r;
    eS[tid] = a.Bexp[t * tc::NT + tid];
  }
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < TC_STAGES; ++i) {
      tc::mbar_init(&mb_tma[i], 1);
      tc::mbar_init(&mb_mma[i], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_slot;
  // the operator box of this tile (per-box operators: every column shares it)
  const int box_op = s.shared ? 0 : max(0, boxof[0]);
  const int mrow = mt * tc::MT + (warp & 3) * 32 + lane;     // operator row of this thread's TMEM lane
  const int chalf = warp >> 2;                                // columns chalf * 16 .. + 15
  // bulk copies of global step g (pole pbeg + g / nk, K step g % nk) into stage g % TC_STAGES
  auto issue_copy = [&](int g) -> bool {
    const int st = g % TC_STAGES, use = g / TC_STAGES;
    if (use > 0 && !tc::mbar_wait(&mb_mma[st], (use - 1) & 1, TC_SPIN)) return false;
    const int pl = pbeg + g / nk, ks = g % nk;
    const int p = s.p0 + pl;
    const bool src = ks < a.nks;
    uint8_t* sa = tsm + (size_t)st * SB;
    const uint8_t* ga = (const uint8_t*)a.Aop +
                        ((((size_t)p * a.nbox_op + box_op) * 2 + mt) * nk + ks) * (size_t)(2 * S * tc::A_BLK);
    tc::mbar_expect_tx(&mb_tma[st], 2 * S * tc::A_BLK + (src ? S * tc::B_BLK : 0));
    tc::bulk_g2s(sa, ga, 2 * S * tc::A_BLK, &mb_tma[st]);
    if (src) {
      const uint8_t* gb = (const uint8_t*)a.Bs + ((size_t)t * a.nks + ks) * (size_t)(S * tc::B_BLK);
      tc::bulk_g2s(sa + 2 * S * tc::A_BLK, gb, S * tc::B_BLK, &mb_tma[st]);
    }
    return true;
  };
  if (tid == 0)
    for (int g = 0; g < min(TC_AHEAD, total); ++g)
      if (!issue_copy(g)) s_abort = 1;
  // per-thread pole-sum accumulators: 16 columns x K weights, FP32 pairs
  float acc[16][3][2];
#pragma unroll
  for (int c = 0; c < 16; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[c][k][0] = acc[c][k][1] = 0.0f;
  bool first[12];
  for (int it = 0; it < npole && !s_abort; ++it) {
    const int pl = pbeg + it, p = s.p0 + pl;
    // edge-block column exponents of this pole (warp w: columns 4w .. 4w + 3)
    for (int n = warp * 4; n < warp * 4 + 4; ++n) {
      const int box = boxof[n], r = rof[n];
      double m = 0.0;
      if (box >= 0)
        for (int j = lane; j < nb; j += 32) {
          const cd v = a.E[((long long)pl * s.R + r) * s.n_edge + (long long)a.bseg[box * 4 + j / q] * q + (j % q)];
          m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
        }
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) eE[n] = tc::split_exponent(m);
    }
    if (tid < K) {
      const cd w = s.wgt[p * K + tid];
      const float wrh = __double2float_rn(w.x), wih = __double2float_rn(w.y);
      wdf[tid][0] = wrh;
      wdf[tid][1] = __double2float_rn(w.x - (double)wrh);
      wdf[tid][2] = wih;
      wdf[tid][3] = __double2float_rn(w.y - (double)wih);
    }
    for (int i = 0; i < 12; ++i) first[i] = true;
    const int* ax = a.Aexp + (((size_t)p * a.nbox_op + box_op) * 2 + mt) * 2 * tc::MT;
    const int erow_s = ax[(warp & 3) * 32 + lane], erow_e = ax[tc::MT + (warp & 3) * 32 + lane];
    __syncthreads();
    for (int ks = 0; ks < nk; ++ks) {
      const int g = it * nk + ks, st = g % TC_STAGES, use = g / TC_STAGES;
      uint8_t* sa = tsm + (size_t)st * SB;
      __nv_bfloat16* sb = (__nv_bfloat16*)(sa + 2 * S * tc::A_BLK);
      const bool src = ks < a.nks;
      if (!src) {
        // edge block of this K step, split per column: 16 K rows x NT columns
        float sr[S], si[S];
        for (int e = tid; e < tc::KS * tc::NT; e += blockDim.x) {
          const int n = e % tc::NT, k = e / tc::NT, j = (ks - a.nks) * tc::KS + k;
          const int box = boxof[n], r = rof[n];
          cd v = make_double2(0.0, 0.0);
          if (box >= 0 && j < nb)
            v = a.E[((long long)pl * s.R + r) * s.n_edge + (long long)a.bseg[box * 4 + j / q] * q + (j % q)];
          tc::split_value<S>(v.x, eE[n], sr);
          tc::split_value<S>(v.y, eE[n], si);
          const int o = tc::core_off(n, k);
#pragma unroll
          for (int i = 0; i < S; ++i) {
            sb[(size_t)i * (tc::B_BLK / 2) + o] = __float2bfloat16_rn(sr[i]);
            sb[(size_t)(S + i) * (tc::B_BLK / 2) + o] = __float2bfloat16_rn(si[i]);
          }
        }
      }
      tc::fence_async_smem();
      __syncthreads();
      if (s_abort) break;
      if (tid == 0) {
        if (!tc::mbar_wait(&mb_tma[st], use & 1, TC_SPIN)) {
          s_abort = 1;
        } else {
          tc::tc_fence_after();
          const uint32_t abase = tc::smem_u32(sa), bbase = tc::smem_u32(sb);
          const uint32_t id0 = tc::idesc_bf16(tc::MT, tc::NT, 0), id1 = tc::idesc_bf16(tc::MT, tc::NT, 1);
          auto mma = [&](int acc_i, int aslot, int bslot, uint32_t idesc) {
            const uint64_t ad = tc::sdesc(abase + aslot * tc::A_BLK, 128, 256);
            const uint64_t bd = tc::sdesc(bbase + bslot * tc::B_BLK, 128, 256);
            tc::mma_bf16(tbase + acc_i * tc::NT, ad, bd, idesc, first[acc_i] ? 0u : 1u);
            first[acc_i] = false;
          };
          for (int i = 1; i <= S; ++i)
            for (int j = 1; i + j <= S + 1; ++j) {
              const int lv = i + j == 2 ? 0 : (i + j == 3 ? 1 : 2);
              if (src) {
                mma(lv * 2 + 0, i - 1, j - 1, id0);
                mma(lv * 2 + 1, S + i - 1, j - 1, id0);
              } else {
                const int re = 6 + lv * 2, im = 7 + lv * 2;
                mma(re, i - 1, j - 1, id0);
                mma(re, S + i - 1, S + j - 1, id1);   // - Im(A) Im(B)
                mma(im, i - 1, S + j - 1, id0);
                mma(im, S + i - 1, j - 1, id0);
              }
            }
          tc::mma_commit(&mb_mma[st]);
          if (g + TC_AHEAD < total && !issue_copy(g + TC_AHEAD)) s_abort = 1;
        }
      }
    }
    // the pole's products are complete when the commit of its last step arrives
    const int gl = it * nk + nk - 1;
    if (!s_abort && !tc::mbar_wait(&mb_mma[gl % TC_STAGES], (gl / TC_STAGES) & 1, TC_SPIN)) s_abort = 1;
    __syncthreads();
    if (s_abort) break;
    tc::tc_fence_after();
    // epilogue: x = 2^(er + ec) (level sums) per block; acc_k += Re(w_pk x)
    const uint32_t lane_base = tbase + ((uint32_t)((warp & 3) * 32) << 16) + chalf * 16;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float v[12][8];
#pragma unroll
      for (int ai = 0; ai < 12; ++ai) {
        uint32_t r8[8];
        const uint32_t ta = lane_base + ai * tc::NT + half * 8;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r8[0]), "=r"(r8[1]), "=r"(r8[2]), "=r"(r8[3]), "=r"(r8[4]), "=r"(r8[5]), "=r"(r8[6]),
                       "=r"(r8[7])
                     : "r"(ta));
#pragma unroll
        for (int c = 0; c < 8; ++c) v[ai][c] = __uint_as_float(r8[c]);
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int n = chalf * 16 + half * 8 + c;
        float xrh, xrl, xih, xil, yh, yl;
        levels(v[0][c], v[2][c], v[4][c], erow_s + eS[n], xrh, xrl);
        levels(v[1][c], v[3][c], v[5][c], erow_s + eS[n], xih, xil);
        levels(v[6][c], v[8][c], v[10][c], erow_e + eE[n], yh, yl);
        df_add(xrh, xrl, yh, yl);
        levels(v[7][c], v[9][c], v[11][c], erow_e + eE[n], yh, yl);
        df_add(xih, xil, yh, yl);
        const int cc = half * 8 + c;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (k >= K) break;
          float ph, plo;
          df_mul(wdf[k][0], wdf[k][1], xrh, xrl, ph, plo);
          df_add(acc[cc][k][0], acc[cc][k][1], ph, plo);
          df_mul(wdf[k][2], wdf[k][3], xih, xil, ph, plo);
          df_add(acc[cc][k][0], acc[cc][k][1], -ph, -plo);
        }
      }
    }
    tc::tc_fence_before();
    __syncthreads();
  }
  // partial sums of this pole chunk
  if (!s_abort && mrow < ni) {
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) {
      const int n = chalf * 16 + cc, box = boxof[n], r = rof[n];
      if (box < 0) continue;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (k >= K) break;
        a.part[(((long long)chunk * s.R + r) * K + k) * s.n_int + (long long)box * ni + mrow] =
            (double)acc[cc][k][0] + (double)acc[cc][k][1];
      }
    }
  }
  if (s_abort) {
    // let every product and copy this block started finish before TMEM is released
    if (tid == 0) {
      atomicExch(a.status, 1);
      for (int st = 0; st < TC_STAGES; ++st) {
        tc::mbar_wait(&mb_mma[st], 0, TC_SPIN >> 4);
        tc::mbar_wait(&mb_tma[st], 0, TC_SPIN >> 4);
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

// ---------------------------------------------------------------- host side
namespace {
constexpr int TC_S = 5;   // slices per real value (about 34 bits kept, ~1e-10 per product)

int tc_tiles(const Handle& h, int R) {
  const int nleaf = h.g.nlx * h.g.nly;
  return h.shared ? (nleaf * R + tc::NT - 1) / tc::NT : nleaf * ((R + tc::NT - 1) / tc::NT);
}
}  // namespace

bool tc_eligible(const Handle& h, std::string* why) {
  const int q = h.g.q, ni = q * q, nb = 4 * q;
  auto no = [&](const char* m) { if (why) *why = m; return false; };
  if (h.fd) return no("the fast-diagonal leaf solves are in use (dense leaves needed)");
  if (h.opts.precision != EO_PREC_DF32) return no("tensor-core leaves need EO_PREC_DF32");
  if (h.K > 3) return no("more than three accumulation weights");
  if (ni > 2 * tc::MT) return no("more than 256 interior nodes per leaf (p > 18)");
  if (nb > 4 * tc::KS) return no("more than 64 edge nodes per leaf (p > 18)");
  return true;
}

// Split the dense leaf operators (FP64, before any reduced-precision copy replaces
// them) into the tensor-core layout; workspace for the per-step source split.
eo_status tc_build(Handle& h, cudaStream_t st) {
  const int q = h.g.q, ni = q * q, nb = 4 * q;
  const int nleaf = h.g.nlx * h.g.nly;
  const int nbox_op = h.shared ? 1 : nleaf;
  h.tc_nks = (h.K * ni + tc::KS - 1) / tc::KS;
  h.tc_nke = (nb + tc::KS - 1) / tc::KS;
  const int nk = h.tc_nks + h.tc_nke;
  const size_t per_op = (size_t)2 * nk * 2 * TC_S * tc::A_BLK;   // bytes per (pole, box): 2 M tiles
  eo_status rc;
  if ((rc = h.alloc((void**)&h.tc_A, per_op * h.P * nbox_op, true))) return rc;
  if ((rc = h.alloc((void**)&h.tc_Aexp, sizeof(int) * (size_t)h.P * nbox_op * 2 * 2 * tc::MT, true))) return rc;
  const int tiles = tc_tiles(h, h.R);
  if ((rc = h.alloc((void**)&h.tc_B, (size_t)tiles * h.tc_nks * TC_S * tc::B_BLK, false))) return rc;
  if ((rc = h.alloc((void**)&h.tc_Bexp, sizeof(int) * (size_t)tiles * tc::NT, false))) return rc;
  if ((rc = h.alloc((void**)&h.tc_status, sizeof(int), false))) return rc;
  EO_CUDA_TRY(cudaMemsetAsync(h.tc_status, 0, sizeof(int), st));
  // pole groups bounded to ~64k blocks per launch
  const int G = std::max(1, std::min(h.P, 65536 / (2 * nbox_op)));
  for (int p0 = 0; p0 < h.P; p0 += G) {
    const int g = std::min(G, h.P - p0);
    k_tc_split_operator<TC_S><<<2 * nbox_op * g, 128, 0, st>>>(
        ni, nb, h.K, h.tc_nks, h.tc_nke, nbox_op, p0, h.XY + (size_t)p0 * h.xy_pstride, h.xy_pstride, h.xy_bstride,
        h.coef, (__nv_bfloat16*)h.tc_A, h.tc_Aexp);
    EO_CUDA_TRY(cudaGetLastError());
  }
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  h.tc = TC_S;
  return EO_OK;
}

// Leaf interiors with the pole sum on the tensor cores: the source split of this
// call's right-hand sides, then the products over poles [s.p0, s.p0 + s.P).
eo_status tc_down_leaf(Handle& h, const Sweep& s, int& nchunk, cudaStream_t st) {
  const int nleaf = h.g.nlx * h.g.nly;
  const int tiles = tc_tiles(h, s.R);
  k_tc_split_sources<TC_S><<<tiles, 256, 0, st>>>(s, nleaf, h.tc_nks, (__nv_bfloat16*)h.tc_B, h.tc_Bexp);
  EO_CUDA_TRY(cudaGetLastError());
  // enough pole chunks for two blocks per SM, at most one chunk per pole
  nchunk = std::max(1, std::min(std::min(s.P, h.nchunk), (2 * 152 + 2 * tiles - 1) / (2 * tiles)));
  const int ppc = (s.P + nchunk - 1) / nchunk;
  nchunk = (s.P + ppc - 1) / ppc;
  TcArgs a;
  a.s = s;
  a.nleaf = nleaf;
  a.nks = h.tc_nks;
  a.nke = h.tc_nke;
  a.nbox_op = h.shared ? 1 : nleaf;
  a.ppc = ppc;
  a.Aop = (const __nv_bfloat16*)h.tc_A;
  a.Aexp = h.tc_Aexp;
  a.Bs = (const __nv_bfloat16*)h.tc_B;
  a.Bexp = h.tc_Bexp;
  a.E = h.E;
  a.bseg = h.lv[0].bseg;
  a.part = h.part;
  a.status = h.tc_status;
  const size_t smem = (size_t)TC_STAGES * tc_stage_bytes<TC_S>();
  static size_t cap[64] = {};
  eo_status rc = ensure_smem((const void*)k_tc_down_leaf<TC_S>, smem, cap, smem);
  if (rc) return rc;
  k_tc_down_leaf<TC_S><<<dim3(tiles, 2, nchunk), 256, smem, st>>>(a);
  EO_CUDA_TRY(cudaGetLastError());
  return EO_OK;
}

eo_status tc_status(Handle& h, cudaStream_t st, int* out) {
  *out = 0;
  if (!h.tc_status) return EO_OK;
  EO_CUDA_TRY(cudaMemcpyAsync(out, h.tc_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  return EO_OK;
}

}  // namespace eo
