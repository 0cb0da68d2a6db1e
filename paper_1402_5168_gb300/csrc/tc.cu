// Leaf down-solves on the tensor cores (tcgen05, bf16 slices, FP32 accumulation in
// TMEM), with the pole sum fused into the epilogue.
//
// The leaf down-solve of pole p (Section 2.3: interior values from the leaf's
// solution operators) is x_p = X_p g_p + Y_p u_b with g_p = sum_k c_pk s_k, s_k the
// pre-mapped sources of the state and u_b the leaf's edge values of pole p.  Both
// products are complex matrix products over the columns (leaf, right-hand side) of a
// tile.  Every real part is split into S bf16 slices (tc.cuh) with a power-of-two
// scale per operator row and per right-hand-side column, separately for the two
// blocks (X with g, Y with u_b), so that each block keeps its own precision whatever
// the ratio of the blocks' magnitudes.  The operator slices are made at build time;
// g_p is formed per pole in FP32-pair arithmetic from pair copies of the sources (no
// FP64 arithmetic on the hot path) and split in the kernel, as is u_b.
// The products of the slices run as tcgen05.mma (M = 128 operator rows, N = 32
// right-hand-side columns, K = 16), accumulated in TMEM in three levels per block
// and component: i + j = 2, 3 and 4 exactly, i + j = 5 .. S + 1 rounded.  The
// epilogue rescales and sums the levels in FP32 pairs (hi, lo), then adds
// Re(w_pk x_p) for every accumulation weight k into per-thread FP32-pair sums; the
// pole chunk's sums go to the same partial-sum array the other leaf kernels fill.
#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "sweep.cuh"
#include "tc.cuh"

namespace eo {

// ---------------------------------------------------------------- build: operator split
// One block per (pole of the group, operator box, M tile); thread t owns row
// mt * 128 + t of [X | Y] (column-major, ni rows).  K steps 0 .. nks-1 hold X
// (kappa = j < ni), K steps nks .. nks+nke-1 hold Y (j' < nb).  Output per
// (pole, box, M tile, K step): 2S slice blocks (re slices, then im slices); per row
// the split exponents of its X and Y parts.
template <int S>
__global__ void __launch_bounds__(128) k_tc_split_operator(int ni, int nb, int nks, int nke, int nbox_op, int pg0,
                                                            const cd* __restrict__ XY, long long xps, long long xbs,
                                                            __nv_bfloat16* __restrict__ Aop, int* __restrict__ Aexp) {
  const int mt = blockIdx.x % 2, box = (blockIdx.x / 2) % nbox_op, gi = blockIdx.x / (2 * nbox_op);
  const int p = pg0 + gi;
  const int row = mt * tc::MT + threadIdx.x;
  const bool ok = row < ni;
  const cd* A = XY + (long long)gi * xps + (long long)box * xbs;
  double mx = 0.0, my = 0.0;
  if (ok) {
    for (int j = 0; j < ni; ++j) {
      const cd x = A[row + (size_t)j * ni];
      mx = fmax(mx, fmax(fabs(x.x), fabs(x.y)));
    }
    for (int j = 0; j < nb; ++j) {
      const cd x = A[row + (size_t)(ni + j) * ni];
      my = fmax(my, fmax(fabs(x.x), fabs(x.y)));
    }
  }
  const int ex = tc::split_exponent(mx), ey = tc::split_exponent(my);
  const size_t opi = ((size_t)p * nbox_op + box) * 2 + mt;
  Aexp[opi * 2 * tc::MT + threadIdx.x] = ex;
  Aexp[opi * 2 * tc::MT + tc::MT + threadIdx.x] = ey;
  const int nk = nks + nke;
  __nv_bfloat16* out = Aop + opi * (size_t)nk * 2 * S * (tc::A_BLK / 2);
  float sr[S], si[S];
  for (int ks = 0; ks < nk; ++ks) {
    __nv_bfloat16* blk = out + (size_t)ks * 2 * S * (tc::A_BLK / 2);
    const bool xb = ks < nks;
    for (int k = 0; k < tc::KS; ++k) {
      const int j = (xb ? ks : ks - nks) * tc::KS + k;
      cd v = make_double2(0.0, 0.0);
      if (ok && j < (xb ? ni : nb)) v = A[row + (size_t)(xb ? j : ni + j) * ni];
      tc::split_value<S>(v.x, xb ? ex : ey, sr);
      tc::split_value<S>(v.y, xb ? ex : ey, si);
      const int o = tc::core_off(threadIdx.x, k);
#pragma unroll
      for (int i = 0; i < S; ++i) {
        blk[(size_t)i * (tc::A_BLK / 2) + o] = __float2bfloat16_rn(sr[i]);
        blk[(size_t)(S + i) * (tc::A_BLK / 2) + o] = __float2bfloat16_rn(si[i]);
      }
    }
  }
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

// ---------------------------------------------------------------- per step: source pairs
// The K pre-mapped sources of every right-hand side as FP32 pairs (hi, lo),
// out[(r * K + k) * n_int + i]: the only conversion from FP64 on the path.
__global__ void k_tc_source_pairs(Sweep s, float2* __restrict__ out) {
  const long long n = (long long)s.R * s.K * s.n_int;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % s.n_int;
    const int k = (int)((e / s.n_int) % s.K), r = (int)(e / ((long long)s.K * s.n_int));
    const double v = s.src[k][r * s.src_rs[k] + i];
    const float h = __double2float_rn(v);
    out[e] = make_float2(h, __double2float_rn(v - (double)h));
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
// four FP32 levels (the first three exact) summed into a pair, times 2^e
__device__ __forceinline__ void levels(float a2, float a3, float a4, float a5, int e, float& h, float& l) {
  two_sum(a2, a3, h, l);
  df_add(h, l, a4, 0.0f);
  df_add(h, l, a5, 0.0f);
  h = ldexpf(h, e);
  l = ldexpf(l, e);
}

struct TcArgs {
  Sweep s;
  int nleaf, nks, nke, nbox_op, ppc;
  const __nv_bfloat16* Aop;   // [P][nbox_op][2 M tiles][nk][2S][MT x KS]
  const int* Aexp;            // [P][nbox_op][2 M tiles][2][MT]
  const float2* srcp;         // sources as pairs [R][K][n_int]
  const cd* E;                // [pole in call][R][n_edge]
  const int* bseg;            // [nleaf][4]
  double* part;               // [chunk][R][K][n_int]
  int* status;                // set to 1 when a bounded wait gives up
};

constexpr int TC_STAGES = 3;
constexpr int TC_AHEAD = 2;          // operator copies issued this many K steps ahead
constexpr int TC_LV = 4;             // accumulator levels: i + j = 2, 3, 4 exact, >= 5 rounded
constexpr int TC_ACC = 2 * 2 * TC_LV;   // per block (X g, Y u_b) and component
constexpr long long TC_SPIN = 1LL << 20;

template <int S>
__host__ __device__ constexpr int tc_stage_bytes() { return 2 * S * (tc::A_BLK + tc::B_BLK); }

// g = sum_k c_k s_k at interior node j of column (box, r), in FP32 pairs (c complex
// pairs cdf[k] = {re hi, re lo, im hi, im lo}, s real pairs)
__device__ __forceinline__ void source_g(const TcArgs& a, const float (*cdf)[4], int box, int r, int j, float& grh,
                                         float& grl, float& gih, float& gil) {
  grh = grl = gih = gil = 0.0f;
  const Sweep& s = a.s;
  for (int k = 0; k < s.K; ++k) {
    const float2 v = a.srcp[((long long)r * s.K + k) * s.n_int + (long long)box * s.ni + j];
    float h, l;
    df_mul(cdf[k][0], cdf[k][1], v.x, v.y, h, l);
    df_add(grh, grl, h, l);
    df_mul(cdf[k][2], cdf[k][3], v.x, v.y, h, l);
    df_add(gih, gil, h, l);
  }
}

// B slices of K step ks for the tile's NT columns into sb: X steps take g (split
// relative to the column's eG), Y steps the edge values u_b (relative to eE).
template <int S>
__device__ __forceinline__ void produce_b(const TcArgs& a, int ks, int pl, const int* boxof, const int* rof,
                                          const int* eG, const int* eE, const float (*cdf)[4],
                                          __nv_bfloat16* sb) {
  const Sweep& s = a.s;
  float sr[S], si[S];
  // producers: warps 1 .. 7 (warp 0 issues the copies and the products)
  for (int e = threadIdx.x - 32; e < tc::KS * tc::NT; e += blockDim.x - 32) {
    const int k = e % tc::KS, n = e / tc::KS;   // consecutive threads: consecutive nodes of a column
    const int box = boxof[n], r = rof[n];
    if (ks < a.nks) {
      const int j = ks * tc::KS + k;
      float grh = 0.f, grl = 0.f, gih = 0.f, gil = 0.f;
      if (box >= 0 && j < s.ni) source_g(a, cdf, box, r, j, grh, grl, gih, gil);
      tc::split_pair_rn<S>(grh, grl, eG[n], sr);
      tc::split_pair_rn<S>(gih, gil, eG[n], si);
    } else {
      const int j = (ks - a.nks) * tc::KS + k;
      cd v = make_double2(0.0, 0.0);
      if (box >= 0 && j < s.nb)
        v = a.E[((long long)pl * s.R + r) * s.n_edge + (long long)a.bseg[box * 4 + j / s.q] * s.q + (j % s.q)];
      tc::split_value<S>(v.x, eE[n], sr);
      tc::split_value<S>(v.y, eE[n], si);
    }
    const int o = tc::core_off(n, k);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      sb[(size_t)i * (tc::B_BLK / 2) + o] = __float2bfloat16_rn(sr[i]);
      sb[(size_t)(S + i) * (tc::B_BLK / 2) + o] = __float2bfloat16_rn(si[i]);
    }
  }
}

// Grid (right-hand-side tiles, 2 M tiles, pole chunks), 256 threads, one block per SM
// (TMEM: TC_ACC = 16 accumulators of NT columns, all 512 columns; shared memory:
// TC_STAGES stages of operator and right-hand-side slices).
template <int S>
__global__ void __launch_bounds__(256, 1) k_tc_down_leaf(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ __align__(8) uint64_t mb_tma[TC_STAGES], mb_mma[TC_STAGES];
  __shared__ uint32_t tmem_slot;
  __shared__ int eG[tc::NT], eE[tc::NT], boxof[tc::NT], rof[tc::NT];
  __shared__ float wdf[3][4], cdf[3][4];
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
  const int box_op = s.shared ? 0 : max(0, boxof[0]);        // per-box operators: every column shares it
  const int mrow = mt * tc::MT + (warp & 3) * 32 + lane;     // operator row of this thread's TMEM lane
  const int chalf = warp >> 2;                                // columns chalf * 16 .. + 15
  // operator slices of global step g (pole pbeg + g / nk, K step g % nk) into stage g % TC_STAGES
  auto issue_copy = [&](int g) -> bool {
    const int st = g % TC_STAGES, use = g / TC_STAGES;
    if (use > 0 && !tc::mbar_wait(&mb_mma[st], (use - 1) & 1, TC_SPIN)) return false;
    const int p = s.p0 + pbeg + g / nk, ks = g % nk;
    const uint8_t* ga = (const uint8_t*)a.Aop +
                        ((((size_t)p * a.nbox_op + box_op) * 2 + mt) * nk + ks) * (size_t)(2 * S * tc::A_BLK);
    tc::mbar_expect_tx(&mb_tma[st], 2 * S * tc::A_BLK);
    tc::bulk_g2s(tsm + (size_t)st * SB, ga, 2 * S * tc::A_BLK, &mb_tma[st]);
    return true;
  };
  if (tid == 0)
    for (int g = 0; g < min(TC_AHEAD, total); ++g)
      if (!issue_copy(g)) s_abort = 1;
  float acc[16][3][2];   // pole sums: 16 columns x K weights, FP32 pairs
#pragma unroll
  for (int c = 0; c < 16; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[c][k][0] = acc[c][k][1] = 0.0f;
  bool first[TC_ACC];
  for (int it = 0; it < npole && !s_abort; ++it) {
    const int pl = pbeg + it, p = s.p0 + pl;
    if (tid < tc::NT) eG[tid] = INT_MIN / 2;
    if (tid < K) {
      const cd w = s.wgt[p * K + tid], c = s.coef[p * K + tid];
      float h = __double2float_rn(w.x);
      wdf[tid][0] = h;
      wdf[tid][1] = __double2float_rn(w.x - (double)h);
      h = __double2float_rn(w.y);
      wdf[tid][2] = h;
      wdf[tid][3] = __double2float_rn(w.y - (double)h);
      h = __double2float_rn(c.x);
      cdf[tid][0] = h;
      cdf[tid][1] = __double2float_rn(c.x - (double)h);
      h = __double2float_rn(c.y);
      cdf[tid][2] = h;
      cdf[tid][3] = __double2float_rn(c.y - (double)h);
    }
    __syncthreads();
    // split exponents of this pole's columns: g over the interior, u_b over the edges
    {
      const int n = tid / 8, box = boxof[n], r = rof[n];   // 8 threads per column, consecutive nodes
      float m = 0.0f;
      if (box >= 0)
        for (int j = tid % 8; j < ni; j += 8) {
          // an FP32 estimate of g suffices for the scale (digits stay within 64)
          float gr = 0.f, gi = 0.f;
          for (int k = 0; k < K; ++k) {
            const float v = a.srcp[((long long)r * K + k) * s.n_int + (long long)box * ni + j].x;
            gr = __fmaf_rn(cdf[k][0], v, gr);
            gi = __fmaf_rn(cdf[k][2], v, gi);
          }
          m = fmaxf(m, fmaxf(fabsf(gr), fabsf(gi)));
        }
      atomicMax(&eG[n], tc::split_exponent_f(m));
    }
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
    for (int i = 0; i < TC_ACC; ++i) first[i] = true;
    const int* ax = a.Aexp + (((size_t)p * a.nbox_op + box_op) * 2 + mt) * 2 * tc::MT;
    const int erow_x = ax[(warp & 3) * 32 + lane], erow_y = ax[tc::MT + (warp & 3) * 32 + lane];
    __syncthreads();
    if (tid < tc::NT && eG[tid] < -200) eG[tid] = 0;   // a zero column: any scale
    __syncthreads();
    for (int ks = 0; ks < nk; ++ks) {
      const int g = it * nk + ks, st = g % TC_STAGES, use = g / TC_STAGES;
      uint8_t* sa = tsm + (size_t)st * SB;
      __nv_bfloat16* sb = (__nv_bfloat16*)(sa + 2 * S * tc::A_BLK);
      if (warp > 0) produce_b<S>(a, ks, pl, boxof, rof, eG, eE, cdf, sb);
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
          const int blk = ks < a.nks ? 0 : 2 * TC_LV;   // accumulator set of this block
          // descriptors of slot 0; a slot's start address adds its offset / 16 to the
          // 14-bit address field (shared addresses stay below 2^18, so no carry)
          const uint64_t ad0 = tc::sdesc(abase, 128, 256), bd0 = tc::sdesc(bbase, 128, 256);
#pragma unroll
          for (int i = 1; i <= S; ++i)
#pragma unroll
            for (int j = 1; j <= S; ++j) {
              if (i + j > S + 1) continue;
              const int lv = min(i + j - 2, TC_LV - 1);
              const int re = blk + lv * 2, im = re + 1;
              const uint64_t ar = ad0 + (uint64_t)((i - 1) * (tc::A_BLK >> 4));
              const uint64_t ai = ad0 + (uint64_t)((S + i - 1) * (tc::A_BLK >> 4));
              const uint64_t br = bd0 + (uint64_t)((j - 1) * (tc::B_BLK >> 4));
              const uint64_t bi = bd0 + (uint64_t)((S + j - 1) * (tc::B_BLK >> 4));
              tc::mma_bf16(tbase + re * tc::NT, ar, br, id0, first[re] ? 0u : 1u);
              first[re] = false;
              tc::mma_bf16(tbase + re * tc::NT, ai, bi, id1, 1u);   // - Im(A) Im(B)
              tc::mma_bf16(tbase + im * tc::NT, ar, bi, id0, first[im] ? 0u : 1u);
              first[im] = false;
              tc::mma_bf16(tbase + im * tc::NT, ai, br, id0, 1u);
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
    // epilogue: x = 2^(e_row + e_col) (level sums) per block; acc_k += Re(w_pk x)
    const uint32_t lane_base = tbase + ((uint32_t)((warp & 3) * 32) << 16) + chalf * 16;
#pragma unroll
    for (int quarter = 0; quarter < 4; ++quarter) {
      float v[TC_ACC][4];
#pragma unroll
      for (int ai = 0; ai < TC_ACC; ++ai) {
        uint32_t r4[4];
        const uint32_t ta = lane_base + ai * tc::NT + quarter * 4;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r4[0]), "=r"(r4[1]), "=r"(r4[2]), "=r"(r4[3])
                     : "r"(ta));
#pragma unroll
        for (int c = 0; c < 4; ++c) v[ai][c] = __uint_as_float(r4[c]);
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int n = chalf * 16 + quarter * 4 + c;
        // accumulator index: block * 2 TC_LV + level * 2 + component
        float xrh, xrl, xih, xil, yh, yl;
        levels(v[0][c], v[2][c], v[4][c], v[6][c], erow_x + eG[n], xrh, xrl);
        levels(v[1][c], v[3][c], v[5][c], v[7][c], erow_x + eG[n], xih, xil);
        levels(v[8][c], v[10][c], v[12][c], v[14][c], erow_y + eE[n], yh, yl);
        df_add(xrh, xrl, yh, yl);
        levels(v[9][c], v[11][c], v[13][c], v[15][c], erow_y + eE[n], yh, yl);
        df_add(xih, xil, yh, yl);
        const int cc = quarter * 4 + c;
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
  if (s_abort && tid == 0) {
    // let the products and copies this block started finish before TMEM is released
    atomicExch(a.status, 1);
    for (int st = 0; st < TC_STAGES; ++st) {
      tc::mbar_wait(&mb_mma[st], 0, TC_SPIN >> 4);
      tc::mbar_wait(&mb_tma[st], 0, TC_SPIN >> 4);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
}

// ---------------------------------------------------------------- host side
namespace {
constexpr int TC_S = 6;   // slices per real value: 41 bits kept

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

// Split the dense leaf operators [X | Y] (FP64, before any reduced-precision copy
// replaces them) into the tensor-core layout; workspace for the source pairs.
eo_status tc_build(Handle& h, cudaStream_t st) {
  const int q = h.g.q, ni = q * q, nb = 4 * q;
  const int nleaf = h.g.nlx * h.g.nly;
  const int nbox_op = h.shared ? 1 : nleaf;
  h.tc_nks = (ni + tc::KS - 1) / tc::KS;
  h.tc_nke = (nb + tc::KS - 1) / tc::KS;
  const int nk = h.tc_nks + h.tc_nke;
  const size_t per_op = (size_t)2 * nk * 2 * TC_S * tc::A_BLK;   // bytes per (pole, box): 2 M tiles
  eo_status rc;
  if ((rc = h.alloc((void**)&h.tc_A, per_op * h.P * nbox_op, true))) return rc;
  if ((rc = h.alloc((void**)&h.tc_Aexp, sizeof(int) * (size_t)h.P * nbox_op * 2 * 2 * tc::MT, true))) return rc;
  if ((rc = h.alloc((void**)&h.tc_B, sizeof(float2) * (size_t)h.R * h.K * h.g.n_int, false))) return rc;
  if ((rc = h.alloc((void**)&h.tc_status, sizeof(int), false))) return rc;
  EO_CUDA_TRY(cudaMemsetAsync(h.tc_status, 0, sizeof(int), st));
  const int G = std::max(1, std::min(h.P, 65536 / (2 * nbox_op)));   // blocks per launch ~64k
  for (int p0 = 0; p0 < h.P; p0 += G) {
    const int g = std::min(G, h.P - p0);
    k_tc_split_operator<TC_S><<<2 * nbox_op * g, 128, 0, st>>>(ni, nb, h.tc_nks, h.tc_nke, nbox_op, p0,
                                                                  h.XY + (size_t)p0 * h.xy_pstride, h.xy_pstride,
                                                                  h.xy_bstride, (__nv_bfloat16*)h.tc_A, h.tc_Aexp);
    EO_CUDA_TRY(cudaGetLastError());
  }
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  h.tc = TC_S;
  return EO_OK;
}

// Leaf interiors with the pole sum on the tensor cores: the source pairs of this
// call's right-hand sides, then the products over poles [s.p0, s.p0 + s.P).
eo_status tc_down_leaf(Handle& h, const Sweep& s, int& nchunk, cudaStream_t st) {
  const int nleaf = h.g.nlx * h.g.nly;
  const int tiles = tc_tiles(h, s.R);
  const long long nsrc = (long long)s.R * s.K * s.n_int;
  k_tc_source_pairs<<<(unsigned)std::min<long long>(4096, (nsrc + 255) / 256), 256, 0, st>>>(s, (float2*)h.tc_B);
  EO_CUDA_TRY(cudaGetLastError());
  // one wave of blocks (one per SM) when the tiles alone do not fill the GPU
  int sms = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  nchunk = std::max(1, std::min(std::min(s.P, h.nchunk), sms / std::max(1, 2 * tiles)));
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
  a.srcp = (const float2*)h.tc_B;
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
