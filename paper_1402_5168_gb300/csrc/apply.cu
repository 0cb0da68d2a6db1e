// Apply phase: u <- sum_m b_m (tau L - alpha_m)^{-1} u  (Section 1.1, eq. def_RM),
// with the conjugate-pole form of Section 3.3 (one solve per pair), each
// resolvent through the precomputed nested-dissection operators of the build
// (Section 2.3): an upward sweep (leaf particular fluxes, merge-level interface
// corrections) and a downward sweep (interface values, then leaf interiors),
// followed by the weighted pole sum and the recovery of every field from the
// elliptic solution (Section 2.1).
//
// Every level is one launch over (poles x boxes x right-hand sides).  The
// per-box products are complex matrix times (multi-)vector products in FP64:
// operator blocks are column-major and read once per block with coalesced
// 16-byte loads (consecutive threads take consecutive rows), the vectors sit
// in shared memory, and when several columns share a block (shared per-level
// operators, or several right-hand sides) each loaded entry feeds up to 8 of
// them.  The pole sum is accumulated in FP64 in shared memory across the poles
// a block owns and reduced in a fixed order, so results are deterministic.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "fused.cuh"
#include "sweep.cuh"

namespace eo {

// ---------------------------------------------------------------- up: leaves
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_up_leaf(Sweep s, const void* Hv, long long hps,
                                                 long long hbs, int nleaf, cd* __restrict__ h0) {
  extern __shared__ cd smem[];
  const TA* H = (const TA*)Hv;
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int ncols = nleaf * s.R;
  const int c0 = blockIdx.x * NC;
  TA* Bs = (TA*)smem;
  cd* Cs = after(Bs, (size_t)NC * s.ni);
  cd* red = Cs + NC * s.nb;
  int box0, r0;
  col_box(c0, s.R, box0, r0);
  cd cf[3];
  for (int kk = 0; kk < s.K; ++kk) cf[kk] = s.coef[p * s.K + kk];
  for (int e = threadIdx.x; e < NC * s.ni; e += blockDim.x) {
    const int c = e / s.ni, j = e - c * s.ni;
    cd g = make_double2(0.0, 0.0);
    if (c0 + c < ncols) {
      int box, r;
      col_box(c0 + c, s.R, box, r);
      for (int kk = 0; kk < s.K; ++kk) {
        const double v = s.src[kk][r * s.src_rs[kk] + (long long)box * s.ni + j];
        g.x += cf[kk].x * v;
        g.y += cf[kk].y * v;
      }
    }
    Bs[e] = Cv<TA>::from(g);
  }
  __syncthreads();
  const TA* A = H + (long long)p * hps + (s.shared ? 0 : (long long)box0 * hbs);
  cmv<NC, TA>(A, s.nb, s.nb, s.ni, Bs, s.ni, Cs, red);
  for (int e = threadIdx.x; e < NC * s.nb; e += blockDim.x) {
    const int c = e / s.nb, row = e - c * s.nb;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    h0[(((long long)pl * s.R + r) * nleaf + box) * s.nb + row] = Cs[e];
  }
}

// ---------------------------------------------------------------- up: merges
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_up_merge(Sweep s, MergeArgs m, const cd* __restrict__ hin,
                                                  cd* __restrict__ hout) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int ncols = m.nbox * s.R;
  const int c0 = blockIdx.x * NC;
  TA* Bs = (TA*)smem;
  cd* Cs = after(Bs, (size_t)NC * m.n3);
  cd* red = Cs + NC * m.zu_rows;
  for (int e = threadIdx.x; e < NC * m.n3; e += blockDim.x) {
    const int c = e / m.n3, t = e - c * m.n3;
    cd v = make_double2(0.0, 0.0);
    if (c0 + c < ncols) {
      int box, r, ca, cb;
      col_box(c0 + c, s.R, box, r);
      children(m, box, ca, cb);
      const cd* hr = hin + ((long long)pl * s.R + r) * m.nbox_c * m.nbd_c;
      const cd x = hr[(long long)ca * m.nbd_c + m.a3[t]], y = hr[(long long)cb * m.nbd_c + m.b3[t]];
      v = make_double2(x.x + y.x, x.y + y.y);
    }
    Bs[e] = Cv<TA>::from(v);
  }
  __syncthreads();
  int box0, r0;
  col_box(c0, s.R, box0, r0);
  const TA* A = (const TA*)m.ZU + (long long)p * m.zps + (s.shared ? 0 : (long long)box0 * m.zbs);
  cmv<NC, TA>(A, m.zu_rows, m.zu_rows, m.n3, Bs, m.n3, Cs, red);
  for (int e = threadIdx.x; e < NC * m.zu_rows; e += blockDim.x) {
    const int c = e / m.zu_rows, row = e - c * m.zu_rows;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    const cd v = Cs[e];
    if (row < m.n3) {
      m.w3[(((long long)pl * s.R + r) * m.nbox + box) * m.n3 + row] = v;
    } else {
      const int i = row - m.n3;
      int ca, cb;
      children(m, box, ca, cb);
      const cd* hr = hin + ((long long)pl * s.R + r) * m.nbox_c * m.nbd_c;
      const cd x = hr[(long long)(m.par_child[i] ? cb : ca) * m.nbd_c + m.par_idx[i]];
      hout[(((long long)pl * s.R + r) * m.nbox + box) * m.nbd + i] = make_double2(x.x + v.x, x.y + v.y);
    }
  }
}

// Up merge of a reflection-symmetric level: h3 splits into its even and odd parts
// under the interface reversal J (e = (h3 + J h3)/2, o = (h3 - J h3)/2, first halves);
// [-Z; U] h3 = E [-Ze e - Zo o ...]: two products with the (n3/2 + nbd/4) x n3/2 blocks,
// then w3[s] = ye[s] + yo[s], w3[J s] = ye[s] - yo[s] and, on the parent boundary,
// dh[i] = ye[n3/2 + orb i] + osg[i] yo[n3/2 + orb i].
template <int NC, typename TA, int FMT>
__global__ void __launch_bounds__(256) k_up_merge_sym(Sweep s, MergeArgs m, const cd* __restrict__ hin,
                                                      cd* __restrict__ hout) {
  // FMT (FP32-pair blocks only): bit 0, the children's boundary data hin are complex FP32
  // pairs (written so by the level below); bit 1, hout is written as pairs for the level
  // above.  The sums around the block products then stay on the FP32 pipe.
  constexpr bool PIN = (FMT & 1) != 0, POUT = (FMT & 2) != 0;
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int ncols = m.nbox * s.R;
  const int c0 = blockIdx.x * NC;
  const int n3 = m.n3, n3h = m.n3h, rh = m.rh;
  TA* Bs = (TA*)smem;
  cd* Cs = after(Bs, (size_t)NC * n3);
  cd* red = Cs + 2 * NC * rh;
  for (int e = threadIdx.x; e < NC * n3h; e += blockDim.x) {
    const int c = e / n3h, t = e - c * n3h;
    if constexpr (PIN) {
      float4 ev = make_float4(0.f, 0.f, 0.f, 0.f), od = ev;
      if (c0 + c < ncols) {
        int box, r, ca, cb;
        col_box(c0 + c, s.R, box, r);
        children(m, box, ca, cb);
        const float4* hr = reinterpret_cast<const float4*>(hin) + ((long long)pl * s.R + r) * m.nbox_c * m.nbd_c;
        const int tj = n3 - 1 - t;
        const float4 a = cp_add(hr[(long long)ca * m.nbd_c + m.a3[t]], hr[(long long)cb * m.nbd_c + m.b3[t]]);
        const float4 b = cp_add(hr[(long long)ca * m.nbd_c + m.a3[tj]], hr[(long long)cb * m.nbd_c + m.b3[tj]]);
        ev = cp_scale(cp_add(a, b), 0.5f);
        od = cp_scale(cp_add(a, cp_scale(b, -1.0f)), 0.5f);
      }
      Bs[c * n3 + t] = ev;
      Bs[c * n3 + n3h + t] = od;
    } else {
      cd ev = make_double2(0.0, 0.0), od = make_double2(0.0, 0.0);
      if (c0 + c < ncols) {
        int box, r, ca, cb;
        col_box(c0 + c, s.R, box, r);
        children(m, box, ca, cb);
        const cd* hr = hin + ((long long)pl * s.R + r) * m.nbox_c * m.nbd_c;
        const int tj = n3 - 1 - t;
        const cd x1 = hr[(long long)ca * m.nbd_c + m.a3[t]], y1 = hr[(long long)cb * m.nbd_c + m.b3[t]];
        const cd x2 = hr[(long long)ca * m.nbd_c + m.a3[tj]], y2 = hr[(long long)cb * m.nbd_c + m.b3[tj]];
        const double ar = x1.x + y1.x, ai = x1.y + y1.y, br = x2.x + y2.x, bi = x2.y + y2.y;
        ev = make_double2(0.5 * (ar + br), 0.5 * (ai + bi));
        od = make_double2(0.5 * (ar - br), 0.5 * (ai - bi));
      }
      Bs[c * n3 + t] = Cv<TA>::from(ev);
      Bs[c * n3 + n3h + t] = Cv<TA>::from(od);
    }
  }
  __syncthreads();
  const TA* A = (const TA*)m.ZUs + (long long)p * m.zsps;
  cmv<NC, TA, POUT>(A, rh, rh, n3h, Bs, n3, Cs, red);
  cmv<NC, TA, POUT>(A + (long long)rh * n3h, rh, rh, n3h, Bs + n3h, n3, Cs + (size_t)NC * rh, red);
  for (int e = threadIdx.x; e < NC * m.zu_rows; e += blockDim.x) {
    const int c = e / m.zu_rows, row = e - c * m.zu_rows;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    if constexpr (POUT) {
      const float4* Ce = reinterpret_cast<const float4*>(Cs);
      const float4* Co = Ce + (size_t)NC * rh;
      if (row < n3) {
        const int sr = row < n3h ? row : n3 - 1 - row;
        const float4 b = row < n3h ? Co[c * rh + sr] : cp_scale(Co[c * rh + sr], -1.0f);
        m.w3[(((long long)pl * s.R + r) * m.nbox + box) * n3 + row] = cp_to(cp_add(Ce[c * rh + sr], b));
      } else {
        const int i = row - n3;
        const int k = n3h + m.orb[i];
        const float4 b = cp_scale(Co[c * rh + k], (float)m.osg[i]);
        int ca, cb;
        children(m, box, ca, cb);
        const long long xi = ((long long)pl * s.R + r) * m.nbox_c * m.nbd_c +
                             (long long)(m.par_child[i] ? cb : ca) * m.nbd_c + m.par_idx[i];
        const float4 x = PIN ? reinterpret_cast<const float4*>(hin)[xi] : Cv<float4>::from(hin[xi]);
        reinterpret_cast<float4*>(hout)[(((long long)pl * s.R + r) * m.nbox + box) * m.nbd + i] =
            cp_add(x, cp_add(Ce[c * rh + k], b));
      }
    } else {
      const cd* Ce = Cs;
      const cd* Co = Cs + (size_t)NC * rh;
      if (row < n3) {
        const int sr = row < n3h ? row : n3 - 1 - row;
        const double sg = row < n3h ? 1.0 : -1.0;
        const cd a = Ce[c * rh + sr], b = Co[c * rh + sr];
        m.w3[(((long long)pl * s.R + r) * m.nbox + box) * n3 + row] = make_double2(a.x + sg * b.x, a.y + sg * b.y);
      } else {
        const int i = row - n3;
        const int k = n3h + m.orb[i];
        const double sg = (double)m.osg[i];
        const cd a = Ce[c * rh + k], b = Co[c * rh + k];
        int ca, cb;
        children(m, box, ca, cb);
        const long long xi = ((long long)pl * s.R + r) * m.nbox_c * m.nbd_c +
                             (long long)(m.par_child[i] ? cb : ca) * m.nbd_c + m.par_idx[i];
        const cd x = PIN ? cp_to(reinterpret_cast<const float4*>(hin)[xi]) : hin[xi];
        hout[(((long long)pl * s.R + r) * m.nbox + box) * m.nbd + i] =
            make_double2(x.x + a.x + sg * b.x, x.y + a.y + sg * b.y);
      }
    }
  }
}

// Down merge of a reflection-symmetric level: the parent boundary values u enter S
// only through the orbit sums a_r = sum_g u[mem[4r+g]] and b_r = sum_g osg u[mem[4r+g]];
// u3[s] = (Se a)[s] + (So b)[s] + w3[s], u3[J s] = (Se a)[s] - (So b)[s] + w3[J s].
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_down_merge_sym(Sweep s, MergeArgs m, cd* __restrict__ E) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int ncols = m.nbox * s.R;
  const int c0 = blockIdx.x * NC;
  const int n3 = m.n3, n3h = m.n3h, nbq = m.nbq;
  const int q = s.q;
  TA* Bs = (TA*)smem;
  cd* Cs = after(Bs, (size_t)NC * 2 * nbq);
  cd* red = Cs + NC * n3;
  for (int e = threadIdx.x; e < NC * nbq; e += blockDim.x) {
    const int c = e / nbq, r = e - c * nbq;
    cd a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    if (c0 + c < ncols) {
      int box, rr;
      col_box(c0 + c, s.R, box, rr);
      const cd* Er = E + ((long long)pl * s.R + rr) * s.n_edge;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int i = m.mem[4 * r + g];
        const cd v = Er[(long long)m.bseg[box * m.nseg + i / q] * q + (i % q)];
        const double sg = g < 2 ? 1.0 : -1.0;
        a.x += v.x; a.y += v.y;
        b.x += sg * v.x; b.y += sg * v.y;
      }
    }
    Bs[c * 2 * nbq + r] = Cv<TA>::from(a);
    Bs[c * 2 * nbq + nbq + r] = Cv<TA>::from(b);
  }
  __syncthreads();
  const TA* A = (const TA*)m.Ss + (long long)p * m.ssps;
  cmv<NC, TA>(A, n3h, n3h, nbq, Bs, 2 * nbq, Cs, red);
  cmv<NC, TA>(A + (long long)n3h * nbq, n3h, n3h, nbq, Bs + nbq, 2 * nbq, Cs + (size_t)NC * n3h, red);
  const cd* Ce = Cs;
  const cd* Co = Cs + (size_t)NC * n3h;
  const int n3s = n3 / q;
  for (int e = threadIdx.x; e < NC * n3; e += blockDim.x) {
    const int c = e / n3, row = e - c * n3;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    const int sr = row < n3h ? row : n3 - 1 - row;
    const double sg = row < n3h ? 1.0 : -1.0;
    const cd a = Ce[c * n3h + sr], b = Co[c * n3h + sr];
    const cd w = m.w3[(((long long)pl * s.R + r) * m.nbox + box) * n3 + row];
    E[((long long)pl * s.R + r) * s.n_edge + (long long)m.iseg[box * n3s + row / q] * q + (row % q)] =
        make_double2(w.x + a.x + sg * b.x, w.y + a.y + sg * b.y);
  }
}

// ---------------------------------------------------------------- root (walls)
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_root_sw(Sweep s, RootArgs ra, const cd* __restrict__ hroot,
                                                 cd* __restrict__ E) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int c0 = blockIdx.x * NC;
  const int n = ra.n;
  TA* Bs = (TA*)smem;
  cd* Cs = after(Bs, (size_t)NC * n);
  cd* red = Cs + NC * n;
  for (int e = threadIdx.x; e < NC * n; e += blockDim.x) {
    const int c = e / n, i = e - c * n;
    cd v = make_double2(0.0, 0.0);
    const int r = c0 + c;
    if (r < s.R) {
      int side;
      if (i < ra.sxq) side = 0;
      else if (i < ra.sxq + ra.syq) side = 1;
      else if (i < 2 * ra.sxq + ra.syq) side = 2;
      else side = 3;
      const long long node = s.n_int + (long long)ra.bseg[i / ra.q] * ra.q + (i % ra.q);
      const double F1 = ra.state[(long long)r * ra.F * s.n_nodes + node];
      const double F2 = ra.state[((long long)r * ra.F + 1) * s.n_nodes + node];
      const cd b0 = ra.bcoef[(p * 4 + side) * 2], b1 = ra.bcoef[(p * 4 + side) * 2 + 1];
      const cd nu = ra.nu[p * 4 + side];
      const cd hr = hroot[((long long)pl * s.R + r) * n + i];
      const cd nh = cmul(nu, hr);
      v = make_double2(b0.x * F1 + b1.x * F2 - nh.x, b0.y * F1 + b1.y * F2 - nh.y);
    }
    Bs[e] = Cv<TA>::from(v);
  }
  __syncthreads();
  // rows [r_lo, r_lo + nr) of the wall solve (blocks along z split the rows)
  const int rows_per = (n + gridDim.z - 1) / gridDim.z;
  const int r_lo = blockIdx.z * rows_per, nr = min(rows_per, n - r_lo);
  if (nr <= 0) return;
  cmv<NC, TA>((const TA*)ra.Binv + (long long)p * n * n + r_lo, n, nr, n, Bs, n, Cs, red);
  for (int e = threadIdx.x; e < NC * nr; e += blockDim.x) {
    const int c = e / nr, i = r_lo + (e - c * nr);
    const int r = c0 + c;
    if (r >= s.R) continue;
    E[((long long)pl * s.R + r) * s.n_edge + (long long)ra.bseg[i / ra.q] * ra.q + (i % ra.q)] = Cs[e];
  }
}

// Root wall solve on a square walled domain: h_b = B^{-1} v with B = D P^T C P, D the
// per-side row signs c4_sign, P the counterclockwise reordering (c4idx) and C block
// circulant over the four sides.  So h_b = P^T G diag(Chat_m^{-1}) H P D v with
// H: rhat_m = (1/4) sum_k (-i)^{mk} r_k and G: y_k = sum_m i^{mk} yhat_m, and Binv
// holds the four inverse Fourier blocks of each pole (nq x nq, nq = n / 4).
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_root_sw_c4(Sweep s, RootArgs ra, const cd* __restrict__ hroot,
                                                    cd* __restrict__ E) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int c0 = blockIdx.x * NC;
  const int n = ra.n, nq = ra.nq;
  TA* Bs = (TA*)smem;
  cd* Cs = after(Bs, (size_t)NC * n);
  cd* red = Cs + NC * n;
  // wall right-hand side v in wall order (into Cs, free until the products)
  for (int e = threadIdx.x; e < NC * n; e += blockDim.x) {
    const int c = e / n, i = e - c * n;
    cd v = make_double2(0.0, 0.0);
    const int r = c0 + c;
    if (r < s.R) {
      const int side = i / nq;
      const long long node = s.n_int + (long long)ra.bseg[i / ra.q] * ra.q + (i % ra.q);
      const double F1 = ra.state[(long long)r * ra.F * s.n_nodes + node];
      const double F2 = ra.state[((long long)r * ra.F + 1) * s.n_nodes + node];
      const cd b0 = ra.bcoef[(p * 4 + side) * 2], b1 = ra.bcoef[(p * 4 + side) * 2 + 1];
      const cd nu = ra.nu[p * 4 + side];
      const cd hr = hroot[((long long)pl * s.R + r) * n + i];
      const cd nh = cmul(nu, hr);
      v = make_double2(b0.x * F1 + b1.x * F2 - nh.x, b0.y * F1 + b1.y * F2 - nh.y);
    }
    Cs[e] = v;
  }
  __syncthreads();
  // rhat_m[s] = (1/4) sum_k (-i)^{mk} c4_sign(k) v[idx_k(s)]: Bs[c][m * nq + s]
  for (int e = threadIdx.x; e < NC * n; e += blockDim.x) {
    const int c = e / n, rem = e - c * n, m = rem / nq, sr = rem - m * nq;
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const cd v = times_ipow(Cs[c * n + ra.c4idx[k * nq + sr]], -(m * k));
      re += c4_sign(k) * v.x;
      im += c4_sign(k) * v.y;
    }
    Bs[e] = Cv<TA>::from(make_double2(0.25 * re, 0.25 * im));
  }
  __syncthreads();
  // yhat_m = Chat_m^{-1} rhat_m: Cs[m][c][s]
  const TA* A = (const TA*)ra.Binv + (long long)p * 4 * nq * nq;
  for (int m = 0; m < 4; ++m)
    cmv<NC, TA>(A + (long long)m * nq * nq, nq, nq, nq, Bs + m * nq, n, Cs + (size_t)m * NC * nq, red);
  // y_k[s] = sum_m i^{mk} yhat_m[s], stored at wall index idx_k(s)
  for (int e = threadIdx.x; e < NC * n; e += blockDim.x) {
    const int c = e / n, rem = e - c * n, k = rem / nq, sr = rem - k * nq;
    const int r = c0 + c;
    if (r >= s.R) continue;
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const cd v = times_ipow(Cs[((size_t)m * NC + c) * nq + sr], m * k);
      re += v.x;
      im += v.y;
    }
    const int i = ra.c4idx[k * nq + sr];
    E[((long long)pl * s.R + r) * s.n_edge + (long long)ra.bseg[i / ra.q] * ra.q + (i % ra.q)] =
        make_double2(re, im);
  }
}

// Root of a periodic square: the seams are interfaces of the root box with itself.
// With the root's particular fluxes h (boundary order S, E, N, W) the seam values are
// s = -Binv P^T h, P^T adding the two sides that meet at a seam (S with N, W with E);
// they are the edge values of the seam segments (the S and W segments of the root,
// which are also its N and E segments).  ra.n = root boundary nodes, Binv (n/2)^2.
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_root_periodic(Sweep s, RootArgs ra, const cd* __restrict__ hroot,
                                                       cd* __restrict__ E) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int c0 = blockIdx.x * NC;
  const int n = ra.n, m = n / 2, sxq = ra.sxq, syq = ra.syq;
  TA* Bs = (TA*)smem;
  cd* Cs = after(Bs, (size_t)NC * m);
  cd* red = Cs + NC * m;
  for (int e = threadIdx.x; e < NC * m; e += blockDim.x) {
    const int c = e / m, r = e - c * m;
    cd v = make_double2(0.0, 0.0);
    const int rr = c0 + c;
    if (rr < s.R) {
      int i1, i2;
      if (r < sxq) { i1 = r; i2 = sxq + syq + r; }
      else { i1 = 2 * sxq + syq + (r - sxq); i2 = sxq + (r - sxq); }
      const cd* hr = hroot + ((long long)pl * s.R + rr) * n;
      const cd a = hr[i1], b = hr[i2];
      v = make_double2(-(a.x + b.x), -(a.y + b.y));
    }
    Bs[e] = Cv<TA>::from(v);
  }
  __syncthreads();
  // rows [r_lo, r_lo + nr) of the seam solve (blocks along z split the rows)
  const int rows_per = (m + gridDim.z - 1) / gridDim.z;
  const int r_lo = blockIdx.z * rows_per, nr = min(rows_per, m - r_lo);
  if (nr <= 0) return;
  cmv<NC, TA>((const TA*)ra.Binv + (long long)p * m * m + r_lo, m, nr, m, Bs, m, Cs, red);
  for (int e = threadIdx.x; e < NC * nr; e += blockDim.x) {
    const int c = e / nr, r = r_lo + (e - c * nr);
    const int rr = c0 + c;
    if (rr >= s.R) continue;
    const int i = r < sxq ? r : 2 * sxq + syq + (r - sxq);   // the S or W node of seam node r
    E[((long long)pl * s.R + rr) * s.n_edge + (long long)ra.bseg[i / ra.q] * ra.q + (i % ra.q)] = Cs[e];
  }
}

// ---------------------------------------------------------------- down: merges
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_down_merge(Sweep s, MergeArgs m, cd* __restrict__ E) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int ncols = m.nbox * s.R;
  const int c0 = blockIdx.x * NC;
  TA* Bs = (TA*)smem;
  cd* Cs = after(Bs, (size_t)NC * m.nbd);
  cd* red = Cs + NC * m.n3;
  const int q = s.q;
  if (m.S) {
    for (int e = threadIdx.x; e < NC * m.nbd; e += blockDim.x) {
      const int c = e / m.nbd, i = e - c * m.nbd;
      cd v = make_double2(0.0, 0.0);
      if (c0 + c < ncols) {
        int box, r;
        col_box(c0 + c, s.R, box, r);
        v = E[((long long)pl * s.R + r) * s.n_edge + (long long)m.bseg[box * m.nseg + i / q] * q + (i % q)];
      }
      Bs[e] = Cv<TA>::from(v);
    }
    __syncthreads();
    int box0, r0;
    col_box(c0, s.R, box0, r0);
    const TA* A = (const TA*)m.S + (long long)p * m.sps + (s.shared ? 0 : (long long)box0 * m.sbs);
    cmv<NC, TA>(A, m.n3, m.n3, m.nbd, Bs, m.nbd, Cs, red);
  }
  const int n3s = m.n3 / q;
  for (int e = threadIdx.x; e < NC * m.n3; e += blockDim.x) {
    const int c = e / m.n3, row = e - c * m.n3;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    cd v = m.w3[(((long long)pl * s.R + r) * m.nbox + box) * m.n3 + row];
    if (m.S) {
      v.x += Cs[e].x;
      v.y += Cs[e].y;
    }
    E[((long long)pl * s.R + r) * s.n_edge + (long long)m.iseg[box * n3s + row / q] * q + (row % q)] = v;
  }
}

// ---------------------------------------------------------------- down: leaves + pole sum
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_down_leaf(Sweep s, const void* XYv, long long xps,
                                                   long long xbs, const int* __restrict__ bseg, int nleaf,
                                                   int ppc, const cd* __restrict__ E,
                                                   double* __restrict__ part) {
  extern __shared__ cd smem[];
  const int ni = s.ni, nb = s.nb, k = ni + nb, q = s.q;
  const int ncols = nleaf * s.R;
  const int c0 = blockIdx.x * NC;
  const int chunk = blockIdx.y;
  const TA* XY = (const TA*)XYv;
  TA* Bs = (TA*)smem;
  double* acc = (double*)after(Bs, (size_t)NC * k);   // [NC][K][ni], each entry owned by one thread
  for (int e = threadIdx.x; e < NC * s.K * ni; e += blockDim.x) acc[e] = 0.0;
  int box0, r0;
  col_box(c0, s.R, box0, r0);
  const int pbeg = chunk * ppc, pend = min(s.P, pbeg + ppc);
  for (int pl = pbeg; pl < pend; ++pl) {
    const int p = s.p0 + pl;
    cd cf[3];
    for (int kk = 0; kk < s.K; ++kk) cf[kk] = s.coef[p * s.K + kk];
    __syncthreads();
    for (int e = threadIdx.x; e < NC * k; e += blockDim.x) {
      const int c = e / k, j = e - c * k;
      cd v = make_double2(0.0, 0.0);
      if (c0 + c < ncols) {
        int box, r;
        col_box(c0 + c, s.R, box, r);
        if (j < ni) {
          for (int kk = 0; kk < s.K; ++kk) {
            const double x = s.src[kk][r * s.src_rs[kk] + (long long)box * ni + j];
            v.x += cf[kk].x * x;
            v.y += cf[kk].y * x;
          }
        } else {
          const int i = j - ni;
          v = E[((long long)pl * s.R + r) * s.n_edge + (long long)bseg[box * 4 + i / q] * q + (i % q)];
        }
      }
      Bs[e] = Cv<TA>::from(v);
    }
    __syncthreads();
    const TA* A = XY + (long long)p * xps + (s.shared ? 0 : (long long)box0 * xbs);
    cd w[3];
    for (int kk = 0; kk < s.K; ++kk) w[kk] = s.wgt[p * s.K + kk];
    // one row per thread, NC columns in registers; the pole-sum update goes
    // straight from registers to the thread's own entries of acc
    for (int row = threadIdx.x; row < ni; row += blockDim.x) {
      typename Cv<TA>::Acc av[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) av[c] = Cv<TA>::zero();
      const TA* Ar = A + row;
      int j = 0;
      for (; j + 3 < k; j += 4) {
        const TA a0 = operator_ld(Ar + (size_t)j * ni);
        const TA a1 = operator_ld(Ar + (size_t)(j + 1) * ni);
        const TA a2 = operator_ld(Ar + (size_t)(j + 2) * ni);
        const TA a3 = operator_ld(Ar + (size_t)(j + 3) * ni);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          Cv<TA>::mac(av[c], a0, Bs[c * k + j]);
          Cv<TA>::mac(av[c], a1, Bs[c * k + j + 1]);
          Cv<TA>::mac(av[c], a2, Bs[c * k + j + 2]);
          Cv<TA>::mac(av[c], a3, Bs[c * k + j + 3]);
        }
      }
      for (; j < k; ++j) {
        const TA a0 = operator_ld(Ar + (size_t)j * ni);
#pragma unroll
        for (int c = 0; c < NC; ++c) Cv<TA>::mac(av[c], a0, Bs[c * k + j]);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const cd x = Cv<TA>::to(av[c]);
        for (int kk = 0; kk < s.K; ++kk) acc[(c * s.K + kk) * ni + row] += w[kk].x * x.x - w[kk].y * x.y;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NC * s.K * ni; e += blockDim.x) {
    const int c = e / (s.K * ni), rem = e - c * s.K * ni, kk = rem / ni, row = rem - kk * ni;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    part[(((long long)chunk * s.R + r) * s.K + kk) * s.n_int + (long long)box * ni + row] = acc[e];
  }
}

// edge-node pole sums: eacc[r][k][e] = sum_p Re(w[p][k] E_p[r][e]).  A block
// takes 32 consecutive (rhs, edge node) entries; its 8 warps stride over the
// poles (coalesced 32-entry rows of E) and the warp partials are added in a
// fixed order, so the sum is deterministic.
__global__ void __launch_bounds__(256) k_edge_acc(Sweep s, const cd* __restrict__ E, double* __restrict__ eacc) {
  __shared__ double red[8][3][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long long tot = (long long)s.R * s.n_edge;
  const long long t = (long long)blockIdx.x * 32 + lane;
  const bool ok = t < tot;
  const int r = ok ? (int)(t / s.n_edge) : 0;
  const long long e = ok ? t - (long long)r * s.n_edge : 0;
  double a[3] = {0, 0, 0};
  if (ok)
    for (int pl = wp; pl < s.P; pl += 8) {
      const cd x = E[((long long)pl * s.R + r) * s.n_edge + e];
      for (int kk = 0; kk < s.K; ++kk) {
        const cd w = s.wgt[(s.p0 + pl) * s.K + kk];
        a[kk] = fma(w.x, x.x, fma(-w.y, x.y, a[kk]));
      }
    }
  for (int kk = 0; kk < s.K; ++kk) red[wp][kk][lane] = a[kk];
  __syncthreads();
  if (wp == 0 && ok)
    for (int kk = 0; kk < s.K; ++kk) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += red[w][kk][lane];
      eacc[((long long)r * s.K + kk) * s.n_edge + e] = v;
    }
}

// accumulated field kk at node (r) from the chunk partials / edge sums
__device__ __forceinline__ double accum(const Sweep& s, int nchunk, const double* part,
                                        const double* eacc, int r, int kk, long long node) {
  if (node < s.n_int) {
    double v = 0;
    for (int c = 0; c < nchunk; ++c) v += part[(((long long)c * s.R + r) * s.K + kk) * s.n_int + node];
    return v;
  }
  return eacc[((long long)r * s.K + kk) * s.n_edge + (node - s.n_int)];
}

// wave post-map: v = A0, u = A1 - C0 u_in
__global__ void k_post_wave(Sweep s, int nchunk, const double* __restrict__ part,
                            const double* __restrict__ eacc, const double* __restrict__ uin,
                            double* __restrict__ uout, double C0) {
  const long long tot = (long long)s.R * s.n_nodes;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / s.n_nodes);
    const long long node = t - (long long)r * s.n_nodes;
    const double a0 = accum(s, nchunk, part, eacc, r, 0, node);
    const double a1 = accum(s, nchunk, part, eacc, r, 1, node);
    const double u = uin[(long long)r * 2 * s.n_nodes + node];
    uout[(long long)r * 2 * s.n_nodes + node] = a1 - C0 * u;
    uout[((long long)r * 2 + 1) * s.n_nodes + node] = a0;
  }
}

// shallow water: accumulated fields at every node, afull[r][k][node]
__global__ void k_reduce_full(Sweep s, int nchunk, const double* __restrict__ part,
                              const double* __restrict__ eacc, double* __restrict__ afull) {
  const long long tot = (long long)s.R * s.K * s.n_nodes;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long rk = t / s.n_nodes;
    const long long node = t - rk * s.n_nodes;
    const int r = (int)(rk / s.K), kk = (int)(rk % s.K);
    afull[t] = accum(s, nchunk, part, eacc, r, kk, node);
  }
}

// wave pre-map: A u = d/dx(c^2 du/dx) + d/dy(c^2 du/dy) at interior nodes by
// nested leaf differentiation (the collocation rows of Section 2.2), pre[r][n_int]
__global__ void k_pre_wave(LeafGeo g, int R, long long n_nodes, const double* __restrict__ acoef,
                           const double* __restrict__ state, double* __restrict__ pre) {
  const int leaf = blockIdx.x, r = blockIdx.y;
  const int a = leaf % g.nlx, b = leaf / g.nlx, p = g.p, q = g.q;
  extern __shared__ double sd[];
  double* u = sd;
  double* al = sd + p * p;
  double* fx = sd + 2 * p * p;   // a * du/dx at (l, j)
  double* fy = sd + 3 * p * p;   // a * du/dy at (k, l)
  const double* U = state + (long long)r * 2 * n_nodes;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const long long id = gnode(g, a, b, t % p, t / p);
    u[t] = id < 0 ? 0.0 : U[id];
    al[t] = id < 0 ? 0.0 : acoef[id];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int k = t % p, j = t / p;
    double sx = 0, sy = 0;
    for (int m = 0; m < p; ++m) {
      sx += g.Dx[k * p + m] * u[j * p + m];
      sy += g.Dy[j * p + m] * u[m * p + k];
    }
    fx[t] = al[t] * sx;
    fy[t] = al[t] * sy;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) {
    const int k = t % q + 1, j = t / q + 1;
    double s = 0;
    for (int l = 0; l < p; ++l) s += g.Dx[k * p + l] * fx[j * p + l] + g.Dy[j * p + l] * fy[l * p + k];
    pre[(long long)r * g.n_int + (long long)leaf * q * q + t] = s;
  }
}

// shallow-water pre-map: div F and curl F at interior nodes, pre[r][0|1][n_int]
__global__ void k_pre_sw(LeafGeo g, int R, long long n_nodes, const double* __restrict__ state,
                         double* __restrict__ pre) {
  const int leaf = blockIdx.x, r = blockIdx.y;
  const int a = leaf % g.nlx, b = leaf / g.nlx, p = g.p, q = g.q;
  extern __shared__ double sd[];
  double* f1 = sd;
  double* f2 = sd + p * p;
  const double* F1 = state + (long long)r * 3 * n_nodes;
  const double* F2 = F1 + n_nodes;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const long long id = gnode(g, a, b, t % p, t / p);
    f1[t] = id < 0 ? 0.0 : F1[id];
    f2[t] = id < 0 ? 0.0 : F2[id];
  }
  __syncthreads();
  const long long ni = (long long)q * q;
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) {
    const int k = t % q + 1, j = t / q + 1;
    const long long o = (long long)leaf * ni + t;
    pre[((long long)r * 2) * g.n_int + o] = ddx(g, f1, k, j) + ddy(g, f2, k, j);
    pre[((long long)r * 2 + 1) * g.n_int + o] = ddx(g, f2, k, j) - ddy(g, f1, k, j);
  }
}

// shallow-water post-map: h = A0,
//   U = C1 F1 + C2 F2 + tau g (dA1/dx + dA2/dy), V = -C2 F1 + C1 F2 + tau g (-dA2/dx + dA1/dy)
// Interior nodes by leaf differentiation; edge nodes owned by this leaf (S and W,
// plus E / N on the walls of a walled square): normal derivative = mean of the one-sided
// derivatives of the leaves that touch the edge, tangential = edge interpolant.
// Three-field wave form: pre[r][1][i] = v[r][i] / kappa[i] at the interior nodes (the
// source of the elliptic solve; the slot of the curl, which the form does not use).
__global__ void k_pre_kappa(int R, long long n_int, long long n_nodes, const double* __restrict__ state,
                            const double* __restrict__ hw, double* __restrict__ pre) {
  const long long tot = (long long)R * n_int;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / n_int, i = t - r * n_int;
    pre[(2 * r + 1) * n_int + i] = state[(3 * r + 2) * n_nodes + i] * hw[i];
  }
}

__global__ void k_post_sw(LeafGeo g, int R, long long n_nodes, int K, const double* __restrict__ afull,
                          const double* __restrict__ uin, double* __restrict__ uout, double C1, double C2,
                          double taug) {
  const int leaf = blockIdx.x, r = blockIdx.y;
  const int a = leaf % g.nlx, b = leaf / g.nlx, p = g.p, q = g.q;
  extern __shared__ double sd[];
  double* A1 = sd;              // this leaf, p x p
  double* A2 = sd + p * p;
  double* W1 = sd + 2 * p * p;  // west neighbour, p x p
  double* W2 = sd + 3 * p * p;
  double* S1 = sd + 4 * p * p;  // south neighbour, p x p
  double* S2 = sd + 5 * p * p;
  const double* a1g = afull + ((long long)r * K + 1) * n_nodes;
  const double* a2g = afull + ((long long)r * K + 2) * n_nodes;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int k = t % p, j = t / p;
    long long id = gnode(g, a, b, k, j);
    A1[t] = id < 0 ? 0.0 : a1g[id];
    A2[t] = id < 0 ? 0.0 : a2g[id];
    // west / south neighbours (across the seam on a periodic square)
    id = a > 0 ? gnode(g, a - 1, b, k, j) : (g.per ? gnode(g, g.nlx - 1, b, k, j) : -1);
    W1[t] = id < 0 ? 0.0 : a1g[id];
    W2[t] = id < 0 ? 0.0 : a2g[id];
    id = b > 0 ? gnode(g, a, b - 1, k, j) : (g.per ? gnode(g, a, g.nly - 1, k, j) : -1);
    S1[t] = id < 0 ? 0.0 : a1g[id];
    S2[t] = id < 0 ? 0.0 : a2g[id];
  }
  __syncthreads();
  const double* in = uin + (long long)r * 3 * n_nodes;
  double* out = uout + (long long)r * 3 * n_nodes;
  const double* a0g = afull + ((long long)r * K) * n_nodes;
  auto emit = [&](long long id, double d1x, double d1y, double d2x, double d2y) {
    const double F1 = in[id], F2 = in[n_nodes + id];
    out[id] = C1 * F1 + C2 * F2 + taug * (d1x + d2y);
    out[n_nodes + id] = -C2 * F1 + C1 * F2 + taug * (-d2x + d1y);
    out[2 * n_nodes + id] = a0g[id];
  };
  // interior
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) {
    const int k = t % q + 1, j = t / q + 1;
    emit(gnode(g, a, b, k, j), ddx(g, A1, k, j), ddy(g, A1, k, j), ddx(g, A2, k, j), ddy(g, A2, k, j));
  }
  // owned edges
  for (int t = threadIdx.x; t < 4 * q; t += blockDim.x) {
    const int side = t / q, o = t % q + 1;
    // E / N edges are owned by the east / north neighbour (on a periodic square always,
    // the last column's E edge being the first column's W edge)
    if (side == 1 && (g.per || a != g.nlx - 1)) continue;
    if (side == 2 && (g.per || b != g.nly - 1)) continue;
    double d1x, d1y, d2x, d2y;
    long long id;
    if (side == 0 || side == 2) {                // horizontal edge: normal y, tangential x
      const int j = side == 0 ? 0 : p - 1, k = o;
      id = gnode(g, a, b, k, j);
      d1y = ddy(g, A1, k, j);
      d2y = ddy(g, A2, k, j);
      if (side == 0 && (b > 0 || g.per)) {
        d1y = 0.5 * (d1y + ddy(g, S1, k, p - 1));
        d2y = 0.5 * (d2y + ddy(g, S2, k, p - 1));
      }
      d1x = 0; d2x = 0;
      for (int m = 1; m <= q; ++m) {
        d1x += g.Ex[(k - 1) * q + (m - 1)] * A1[j * p + m];
        d2x += g.Ex[(k - 1) * q + (m - 1)] * A2[j * p + m];
      }
    } else {                                     // vertical edge: normal x, tangential y
      const int k = side == 3 ? 0 : p - 1, j = o;
      id = gnode(g, a, b, k, j);
      d1x = ddx(g, A1, k, j);
      d2x = ddx(g, A2, k, j);
      if (side == 3 && (a > 0 || g.per)) {
        d1x = 0.5 * (d1x + ddx(g, W1, p - 1, j));
        d2x = 0.5 * (d2x + ddx(g, W2, p - 1, j));
      }
      d1y = 0; d2y = 0;
      for (int m = 1; m <= q; ++m) {
        d1y += g.Ey[(j - 1) * q + (m - 1)] * A1[m * p + k];
        d2y += g.Ey[(j - 1) * q + (m - 1)] * A2[m * p + k];
      }
    }
    emit(id, d1x, d1y, d2x, d2y);
  }
}

// E[pr][seg * q + o] = 0 for the listed segments (block x: segment, block y: pole x rhs)
__global__ void k_zero_segments(const int* __restrict__ segs, int q, long long n_edge, cd* __restrict__ E) {
  const long long base = (long long)blockIdx.y * n_edge + (long long)segs[blockIdx.x] * q;
  for (int o = threadIdx.x; o < q; o += blockDim.x) E[base + o] = make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------- host driver
namespace {

// Columns per block: with shared operators any columns can share a block, but no
// more than the launch has (nbox * R); with per-box operators the columns of a
// block are right-hand sides of one box, so nc must divide R.
int pick_nc(int shared, int R, int k, int rows, int nbox = 1 << 30) {
  int nc = 1;
  if (shared) {
    const long long ncols = (long long)nbox * R;
    while (nc < 8 && 2 * nc <= ncols) nc *= 2;
  } else {
    while (nc < 8 && R % (nc * 2) == 0) nc *= 2;
  }
  // keep the shared-memory footprint under ~200 KB
  while (nc > 1 && (size_t)nc * (k + rows + 256) * sizeof(cd) > 200 * 1024) nc /= 2;
  return nc;
}

template <template <int, typename> class Launcher, typename TA, typename... Args>
eo_status dispatch_nc(int nc, Args&&... args) {
  switch (nc) {
    case 1: return Launcher<1, TA>::run(args...);
    case 2: return Launcher<2, TA>::run(args...);
    case 4: return Launcher<4, TA>::run(args...);
    default: return Launcher<8, TA>::run(args...);
  }
}

// prec: 0 FP64 blocks, 1 FP32 blocks, 2 FP32-pair blocks
template <template <int, typename> class Launcher, typename... Args>
eo_status dispatch(int prec, int nc, Args&&... args) {
  if (prec == 1) return dispatch_nc<Launcher, float2>(nc, args...);
  if (prec == 2) return dispatch_nc<Launcher, float4>(nc, args...);
  return dispatch_nc<Launcher, double2>(nc, args...);
}

#define EO_SET_SMEM(kern, bytes)                                                            \
  do {                                                                                        \
    /* raise the dynamic shared-memory cap once per kernel and device */                     \
    static size_t cap_[64] = {};                                                              \
    eo_status rs_ = ensure_smem((const void*)(kern), (bytes), cap_, 200 * 1024 + 8192);       \
    if (rs_) return rs_;                                                                      \
  } while (0)

template <int NC, typename TA>
struct UpLeaf {
  static eo_status run(const Sweep& s, const Handle& h, int nleaf, cd* h0, cudaStream_t st) {
    const int ncols = nleaf * s.R;
    dim3 grid((ncols + NC - 1) / NC, s.P);
    const size_t smem = sizeof(cd) * ((size_t)NC * (s.ni + s.nb) + 256 * NC) + 64;
    EO_SET_SMEM((k_up_leaf<NC, TA>), smem);
    k_up_leaf<NC, TA><<<grid, 256, smem, st>>>(s, h.aH, h.h_pstride, h.h_bstride, nleaf, h0);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct UpMerge {
  // fmt: formats of hin / hout for the FP32-pair symmetric kernel (k_up_merge_sym FMT)
  static eo_status run(const Sweep& s, const MergeArgs& m, const cd* hin, cd* hout, int nt, int fmt,
                       cudaStream_t st) {
    dim3 grid((m.nbox * s.R + NC - 1) / NC, s.P);
    const size_t smem = sizeof(cd) * ((size_t)NC * (m.n3 + m.zu_rows) + 256 * NC) + 64;
    if (m.sym) {
      const int thr = nt > 0 ? nt : cmv_threads(m.rh);
      if constexpr (std::is_same<TA, float4>::value) {
        if (fmt == 1) {
          EO_SET_SMEM((k_up_merge_sym<NC, TA, 1>), smem);
          k_up_merge_sym<NC, TA, 1><<<grid, thr, smem, st>>>(s, m, hin, hout);
        } else if (fmt == 2) {
          EO_SET_SMEM((k_up_merge_sym<NC, TA, 2>), smem);
          k_up_merge_sym<NC, TA, 2><<<grid, thr, smem, st>>>(s, m, hin, hout);
        } else if (fmt == 3) {
          EO_SET_SMEM((k_up_merge_sym<NC, TA, 3>), smem);
          k_up_merge_sym<NC, TA, 3><<<grid, thr, smem, st>>>(s, m, hin, hout);
        } else {
          EO_SET_SMEM((k_up_merge_sym<NC, TA, 0>), smem);
          k_up_merge_sym<NC, TA, 0><<<grid, thr, smem, st>>>(s, m, hin, hout);
        }
      } else {
        if (fmt) return fail(EO_ERR_INVALID_ARG, "pair-format boundary data need FP32-pair blocks");
        EO_SET_SMEM((k_up_merge_sym<NC, TA, 0>), smem);
        k_up_merge_sym<NC, TA, 0><<<grid, thr, smem, st>>>(s, m, hin, hout);
      }
      EO_CUDA_TRY(cudaGetLastError());
      return EO_OK;
    }
    if (fmt) return fail(EO_ERR_INVALID_ARG, "pair-format boundary data need the symmetric merge kernel");
    EO_SET_SMEM((k_up_merge<NC, TA>), smem);
    k_up_merge<NC, TA><<<grid, nt > 0 ? nt : cmv_threads(m.zu_rows), smem, st>>>(s, m, hin, hout);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct DownMerge {
  static eo_status run(const Sweep& s, const MergeArgs& m, cd* E, int nt, cudaStream_t st) {
    dim3 grid((m.nbox * s.R + NC - 1) / NC, s.P);
    const size_t smem = sizeof(cd) * ((size_t)NC * (m.nbd + m.n3) + 256 * NC) + 64;
    if (m.sym && m.Ss) {
      EO_SET_SMEM((k_down_merge_sym<NC, TA>), smem);
      k_down_merge_sym<NC, TA><<<grid, nt > 0 ? nt : cmv_threads(m.n3h), smem, st>>>(s, m, E);
      EO_CUDA_TRY(cudaGetLastError());
      return EO_OK;
    }
    EO_SET_SMEM((k_down_merge<NC, TA>), smem);
    k_down_merge<NC, TA><<<grid, nt > 0 ? nt : (m.S ? cmv_threads(m.n3) : 256), smem, st>>>(s, m, E);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct RootSW {
  static eo_status run(const Sweep& s, const RootArgs& ra, const cd* hroot, cd* E, int nt, int rsplit,
                       cudaStream_t st) {
    const size_t smem = sizeof(cd) * ((size_t)NC * 2 * ra.n + 256 * NC) + 64;
    if (ra.nq) {
      dim3 grid((s.R + NC - 1) / NC, s.P, 1);
      EO_SET_SMEM((k_root_sw_c4<NC, TA>), smem);
      k_root_sw_c4<NC, TA><<<grid, nt > 0 ? nt : cmv_threads(ra.nq), smem, st>>>(s, ra, hroot, E);
      EO_CUDA_TRY(cudaGetLastError());
      return EO_OK;
    }
    rsplit = std::max(1, rsplit);
    dim3 grid((s.R + NC - 1) / NC, s.P, rsplit);
    const int rows_per = (ra.n + rsplit - 1) / rsplit;
    EO_SET_SMEM((k_root_sw<NC, TA>), smem);
    k_root_sw<NC, TA><<<grid, nt > 0 ? nt : cmv_threads(rows_per), smem, st>>>(s, ra, hroot, E);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct RootPer {
  static eo_status run(const Sweep& s, const RootArgs& ra, const cd* hroot, cd* E, int nt, int rsplit,
                       cudaStream_t st) {
    const int m = ra.n / 2;
    const size_t smem = sizeof(cd) * ((size_t)NC * 2 * m + 256 * NC) + 64;
    rsplit = std::max(1, rsplit);
    dim3 grid((s.R + NC - 1) / NC, s.P, rsplit);
    const int rows_per = (m + rsplit - 1) / rsplit;
    EO_SET_SMEM((k_root_periodic<NC, TA>), smem);
    k_root_periodic<NC, TA><<<grid, nt > 0 ? nt : cmv_threads(rows_per), smem, st>>>(s, ra, hroot, E);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct DownLeaf {
  static eo_status run(const Sweep& s, const Handle& h, int nleaf, int nchunk, int ppc, const cd* E,
                       double* part, cudaStream_t st) {
    dim3 grid((nleaf * s.R + NC - 1) / NC, nchunk);
    const size_t smem = sizeof(TA) * ((size_t)NC * (s.ni + s.nb)) + sizeof(double) * NC * s.K * s.ni + 64;
    EO_SET_SMEM((k_down_leaf<NC, TA>), smem);
    k_down_leaf<NC, TA><<<grid, 256, smem, st>>>(s, h.aXY, h.xy_pstride, h.xy_bstride, h.lv[0].bseg, nleaf, ppc,
                                            E, part);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

MergeArgs merge_args(const Handle& h, int l) {
  const LevelDev& ld = h.lv[l];
  const LevelDev& lc = h.lv[l - 1];
  MergeArgs m;
  m.nbox = ld.nbox; m.nbx = ld.nbx; m.nbx_c = lc.nbx; m.nbox_c = lc.nbox; m.dir = ld.dir;
  m.nbd = ld.nbd; m.nbd_c = lc.nbd; m.n3 = ld.n3; m.zu_rows = ld.zu_rows;
  m.par_child = ld.par_child; m.par_idx = ld.par_idx; m.a3 = ld.a3; m.b3 = ld.b3;
  m.ZU = ld.aZU; m.zps = ld.zu_pstride; m.zbs = ld.zu_bstride;
  m.S = ld.aS; m.sps = ld.s_pstride; m.sbs = ld.s_bstride;
  m.bseg = ld.bseg; m.iseg = ld.iseg; m.nseg = ld.nseg; m.w3 = ld.w3;
  if (ld.sym) {
    m.sym = 1; m.n3h = ld.n3 / 2; m.rh = ld.rh; m.nbq = ld.rh - ld.n3 / 2;
    m.ZUs = ld.aZUs; m.zsps = ld.zs_pstride; m.Ss = ld.aSs; m.ssps = ld.ss_pstride;
    m.orb = ld.orb; m.osg = ld.osg; m.mem = ld.mem;
  }
  return m;
}

// ---------------------------------------------------------------- fused low levels
// Shared memory of the fused kernels for R right-hand sides (k_up_fused, k_down_fused).
struct FusedSmem {
  size_t up = 0, down = 0;
};

static FusedSmem fused_smem(const FusedLevels& f, int R, int prec) {
  const size_t ta = prec == 1 ? sizeof(float2) : prec == 2 ? sizeof(float4) : sizeof(double2);
  int n3max = 0, rhmax = 0, kmax = 0;
  for (int l = 1; l <= f.Lf; ++l) {
    n3max = std::max(n3max, f.m[l].n3);
    rhmax = std::max(rhmax, f.m[l].rh);
    kmax = std::max(kmax, 2 * f.m[l].nbq);
  }
  FusedSmem z;
  z.up = sizeof(cd) * (2 * (size_t)f.hs + 2 * 8 * rhmax + 256 * 8) + ta * 8 * n3max + 64;
  z.down = sizeof(cd) * ((size_t)8 * n3max + 256 * 8) + ta * 8 * kmax + 64;
  (void)R;
  return z;
}

// Levels 1 .. Lf of both sweeps fused (Lf = 0: none): every level reflection-symmetric
// with even/odd blocks for both sweeps, one block precision, at least one level above,
// and the blocks' shared memory within 200 KB.
FusedLevels fused_plan(const Handle& h, int R) {
  FusedLevels f;
  const int L = h.plan.L();
  const int want = std::min(std::min(h.opts.merge_fuse, FUSED_MAX), L - 1);
  if (want < 1 || !h.shared || h.g.periodic) return f;
  int Lf = 0;
  for (int l = 1; l <= want; ++l) {
    const LevelDev& ld = h.lv[l];
    if (!ld.sym || !ld.aZUs || !ld.aSs || ld.fp32 != h.lv[1].fp32) break;
    Lf = l;
  }
  for (; Lf >= 1; --Lf) {
    f = FusedLevels{};
    f.Lf = Lf;
    for (int l = 0; l <= Lf; ++l) {
      f.nbx[l] = h.lv[l].nbx;
      f.nby[l] = h.lv[l].nbox / h.lv[l].nbx;
      if (l >= 1) f.m[l] = merge_args(h, l);
    }
    const int nsub = h.lv[Lf].nbox;
    f.hs = 0;
    for (int l = 1; l < Lf; ++l)
      f.hs = std::max(f.hs, h.lv[l].nbox / nsub * R * h.lv[l].nbd);
    const FusedSmem z = fused_smem(f, R, h.lv[1].fp32);
    if (std::max(z.up, z.down) <= 200 * 1024) return f;
  }
  return FusedLevels{};
}

// Formats of the boundary data around up level l (k_up_merge_sym FMT): a level run by the
// FP32-pair symmetric kernel writes FP32 pairs when the level above is one too (not the
// root's input, not a fused level); it reads pairs when the level below wrote them.
static bool up_pairs_out(const Handle& h, int l, int Lf) {
  const int L = h.plan.L();
  auto pair_level = [&](int k) { return k > Lf && k <= L && h.lv[k].sym && h.lv[k].fp32 == 2; };
  return l < L && pair_level(l) && pair_level(l + 1);
}
static int up_format(const Handle& h, int l, int Lf) {
  return (l > 1 && up_pairs_out(h, l - 1, Lf) ? 1 : 0) | (up_pairs_out(h, l, Lf) ? 2 : 0);
}

template <typename TA>
static eo_status run_up_fused(const Sweep& s, const FusedLevels& f, const cd* h0, cd* hout, size_t smem,
                              cudaStream_t st) {
  EO_SET_SMEM((k_up_fused<TA>), smem);
  k_up_fused<TA><<<dim3(f.nbx[f.Lf] * f.nby[f.Lf], s.P), 256, smem, st>>>(s, f, h0, hout);
  EO_CUDA_TRY(cudaGetLastError());
  return EO_OK;
}

template <typename TA>
static eo_status run_down_fused(const Sweep& s, const FusedLevels& f, cd* E, size_t smem, cudaStream_t st) {
  EO_SET_SMEM((k_down_fused<TA>), smem);
  k_down_fused<TA><<<dim3(f.nbx[f.Lf] * f.nby[f.Lf], s.P), 256, smem, st>>>(s, f, E);
  EO_CUDA_TRY(cudaGetLastError());
  return EO_OK;
}

static eo_status up_fused(const Handle& h, const Sweep& s, const FusedLevels& f, const cd* h0, cd* hout,
                          cudaStream_t st) {
  const int prec = h.lv[1].fp32;
  const size_t smem = fused_smem(f, s.R, prec).up;
  if (prec == 1) return run_up_fused<float2>(s, f, h0, hout, smem, st);
  if (prec == 2) return run_up_fused<float4>(s, f, h0, hout, smem, st);
  return run_up_fused<double2>(s, f, h0, hout, smem, st);
}

static eo_status down_fused(const Handle& h, const Sweep& s, const FusedLevels& f, cd* E, cudaStream_t st) {
  const int prec = h.lv[1].fp32;
  const size_t smem = fused_smem(f, s.R, prec).down;
  if (prec == 1) return run_down_fused<float2>(s, f, E, smem, st);
  if (prec == 2) return run_down_fused<float4>(s, f, E, smem, st);
  return run_down_fused<double2>(s, f, E, smem, st);
}

Sweep base_sweep(const Handle& h, int R, int p0, int np, const cd* wgt) {
  const Grid& g = h.g;
  Sweep s{};
  s.R = R; s.P = np; s.p0 = p0; s.q = g.q; s.ni = g.q * g.q; s.nb = 4 * g.q;
  s.n_int = g.n_int; s.n_edge = g.n_edge; s.n_nodes = g.n_nodes; s.shared = h.shared;
  s.K = h.K; s.coef = h.coef; s.wgt = wgt;
  return s;
}

LeafGeo leaf_geo(const Handle& h) {
  const Grid& g = h.g;
  const int q = g.q;
  return LeafGeo{g.nlx, g.nly, g.p, q, g.n_int, g.n_hseg, h.dDx, h.dDx + g.p * g.p, h.dDx + 2 * g.p * g.p,
                 h.dDx + 2 * g.p * g.p + q * q, g.periodic};
}

// First part of a step: pre-map, upward sweep, root, downward merges.  Leaves
// every pole's interface and boundary values in h.E and returns the sweep
// description (sources of the leaf solves) in s.
eo_status sweep_to_edges(Handle& h, const double* uin, int R, int p0, int np, const cd* wgt, Sweep& s,
                         cudaStream_t st) {
  const Grid& g = h.g;
  const int q = g.q, ni = q * q, nb = 4 * q;
  const int nleaf = g.nlx * g.nly;
  const int L = h.plan.L();
  eo_status rc;
  s = base_sweep(h, R, p0, np, wgt);
  const LeafGeo geo = leaf_geo(h);
  if (h.kind == EO_WAVE_DIRICHLET) {
    // s = (alpha / tau^2) v + (1 / tau) A u: sources v (field 1) and A u (pre-map)
    if ((rc = h.trace_begin(st))) return rc;
    k_pre_wave<<<dim3(nleaf, R), 128, sizeof(double) * 4 * g.p * g.p, st>>>(geo, R, g.n_nodes, h.acoef, uin,
                                                                          h.pre);
    EO_CUDA_TRY(cudaGetLastError());
    if ((rc = h.trace_end(TR_PRE, st))) return rc;
    s.src[0] = uin + g.n_nodes; s.src_rs[0] = 2 * g.n_nodes;
    s.src[1] = h.pre;           s.src_rs[1] = g.n_int;
  } else {
    if ((rc = h.trace_begin(st))) return rc;
    k_pre_sw<<<dim3(nleaf, R), 128, sizeof(double) * 2 * g.p * g.p, st>>>(geo, R, g.n_nodes, uin, h.pre);
    EO_CUDA_TRY(cudaGetLastError());
    if (h.kappa_form) {
      // three-field wave form: the source of v is v / kappa (the curl slot is free,
      // its coefficient tau f / (g alpha) vanishing with f = 0)
      k_pre_kappa<<<(unsigned)std::min<long long>(4096, (R * g.n_int + 255) / 256), 256, 0, st>>>(
          R, g.n_int, g.n_nodes, uin, h.hw, h.pre);
      EO_CUDA_TRY(cudaGetLastError());
    }
    if ((rc = h.trace_end(TR_PRE, st))) return rc;
    s.src[0] = uin + 2 * g.n_nodes; s.src_rs[0] = 3 * g.n_nodes;
    s.src[1] = h.pre;               s.src_rs[1] = 2 * g.n_int;
    s.src[2] = h.pre + g.n_int;     s.src_rs[2] = 2 * g.n_int;
    if (h.kappa_form) { s.src[0] = h.pre + g.n_int; s.src_rs[0] = 2 * g.n_int; }
  }
  // up: leaves
  cd* hcur = h.hA;
  cd* hnext = h.hB;
  if ((rc = h.trace_begin(st))) return rc;
  if (h.fd) {
    if ((rc = fd_up_leaf(h, s, nleaf, hcur, st))) return rc;
  } else if ((rc = dispatch<UpLeaf>(h.fp32, pick_nc(h.shared, R, ni, nb, nleaf), s, h, nleaf, hcur, st))) {
    return rc;
  }
  if ((rc = h.trace_end(TR_UP_LEAF, st))) return rc;
  // up: merges (the lowest fused into one launch where fused_plan allows)
  const FusedLevels fl = fused_plan(h, R);
  if (fl.Lf) {
    if ((rc = h.trace_begin(st))) return rc;
    if ((rc = up_fused(h, s, fl, hcur, hnext, st))) return rc;
    if ((rc = h.trace_end(TR_UP_MERGE, st))) return rc;
    std::swap(hcur, hnext);
  }
  for (int l = fl.Lf + 1; l <= L; ++l) {
    MergeArgs m = merge_args(h, l);
    if ((rc = h.trace_begin(st))) return rc;
    const Tuned tu = h.lv[l].up;
    const int nc = tu.nc ? tu.nc : pick_nc(h.shared, R, m.n3, m.zu_rows, m.nbox);
    if ((rc = dispatch<UpMerge>(h.lv[l].fp32, nc, s, m, hcur, hnext, tu.nt, up_format(h, l, fl.Lf), st)))
      return rc;
    if ((rc = h.trace_end(TR_UP_MERGE, st))) return rc;
    std::swap(hcur, hnext);
  }
  // root
  if (g.periodic) {
    const Level& rl = h.plan.lv[L];
    RootArgs ra{rl.nbd, q, rl.sx * q, rl.sy * q, h.lv[L].bseg, h.aBinv, nullptr, nullptr, uin, h.F};
    if ((rc = h.trace_begin(st))) return rc;
    const int nc = h.root_tuned.nc ? h.root_tuned.nc : pick_nc(0, R, rl.nbd / 2, rl.nbd / 2);
    if ((rc = dispatch<RootPer>(h.root_fp32, nc, s, ra, hcur, h.E, h.root_tuned.nt, h.root_tuned.rs, st)))
      return rc;
    if ((rc = h.trace_end(TR_ROOT, st))) return rc;
  } else if (h.kind == EO_WAVE_DIRICHLET) {
    // wall values are zero: reset them every step (other users of the edge
    // workspace, such as the adjoint sweeps, leave data there)
    const Level& rl = h.plan.lv[L];
    k_zero_segments<<<dim3(rl.nseg, np * R), 64, 0, st>>>(h.lv[L].bseg, q, g.n_edge, h.E);
    EO_CUDA_TRY(cudaGetLastError());
  } else {
    const Level& rl = h.plan.lv[L];
    RootArgs ra{rl.nbd, q, rl.sx * q, rl.sy * q, h.lv[L].bseg, h.aBinv, h.bcoef, h.nu, uin, 3,
                h.c4, h.c4idx, h.c4inv};
    if ((rc = h.trace_begin(st))) return rc;
    const int nc = h.root_tuned.nc ? h.root_tuned.nc : pick_nc(0, R, rl.nbd, rl.nbd);
    if ((rc = dispatch<RootSW>(h.root_fp32, nc, s, ra, hcur, h.E, h.root_tuned.nt, h.root_tuned.rs, st))) return rc;
    if ((rc = h.trace_end(TR_ROOT, st))) return rc;
  }
  // down: merges
  for (int l = L; l > fl.Lf; --l) {
    MergeArgs m = merge_args(h, l);
    if ((rc = h.trace_begin(st))) return rc;
    const Tuned tu = h.lv[l].down;
    const int nc = tu.nc ? tu.nc : pick_nc(h.shared, R, m.nbd, m.n3, m.nbox);
    if ((rc = dispatch<DownMerge>(h.lv[l].fp32, nc, s, m, h.E, tu.nt, st))) return rc;
    if ((rc = h.trace_end(TR_DOWN_MERGE, st))) return rc;
  }
  if (fl.Lf) {
    if ((rc = h.trace_begin(st))) return rc;
    if ((rc = down_fused(h, s, fl, h.E, st))) return rc;
    if ((rc = h.trace_end(TR_DOWN_MERGE, st))) return rc;
  }
  return EO_OK;
}

// Second part: leaf interiors with the weighted pole sum (weights s.wgt), edge
// sums and the post-map with constants C, into uout.
eo_status finish_step(Handle& h, const Sweep& s, const double* uin, double* uout, const double* C,
                      cudaStream_t st) {
  const Grid& g = h.g;
  const int q = g.q, ni = q * q, nb = 4 * q;
  const int nleaf = g.nlx * g.nly;
  const int R = s.R, np = s.P;
  const LeafGeo geo = leaf_geo(h);
  eo_status rc;
  // down: leaves with the pole sum
  int nchunk = 1;
  if ((rc = h.trace_begin(st))) return rc;
  if (h.fd) {
    if ((rc = fd_down_leaf(h, s, nleaf, h.fd_ncol_down, nchunk, st))) return rc;
  } else if (h.tc) {
    if ((rc = tc_down_leaf(h, s, nchunk, st))) return rc;
  } else {
    const int nc = pick_nc(h.shared, R, ni + nb, ni, nleaf);
    const int ncg = (nleaf * R + nc - 1) / nc;
    nchunk = std::max(1, std::min(np, (608 + ncg - 1) / ncg));
    nchunk = std::min(nchunk, h.nchunk);
    const int ppc = (np + nchunk - 1) / nchunk;
    nchunk = (np + ppc - 1) / ppc;
    if ((rc = dispatch<DownLeaf>(h.fp32, nc, s, h, nleaf, nchunk, ppc, h.E, h.part, st))) return rc;
  }
  if ((rc = h.trace_end(TR_DOWN_LEAF, st))) return rc;
  if ((rc = h.trace_begin(st))) return rc;
  k_edge_acc<<<(unsigned)((R * g.n_edge + 31) / 32), 256, 0, st>>>(s, h.E, h.eacc);
  EO_CUDA_TRY(cudaGetLastError());
  if ((rc = h.trace_end(TR_EDGE, st))) return rc;
  if ((rc = h.trace_begin(st))) return rc;
  if (h.kind == EO_WAVE_DIRICHLET) {
    k_post_wave<<<(unsigned)std::max<long long>(1, std::min<long long>(8192, (R * g.n_nodes + 255) / 256)), 256, 0, st>>>(
        s, nchunk, h.part, h.eacc, uin, uout, C[0]);
    EO_CUDA_TRY(cudaGetLastError());
  } else {
    k_reduce_full<<<(unsigned)std::max<long long>(1, std::min<long long>(8192, (R * 3 * g.n_nodes + 255) / 256)), 256, 0,
                    st>>>(s, nchunk, h.part, h.eacc, h.afull);
    EO_CUDA_TRY(cudaGetLastError());
    k_post_sw<<<dim3(nleaf, R), 128, sizeof(double) * 6 * g.p * g.p, st>>>(
        geo, R, g.n_nodes, h.K, h.afull, uin, uout, C[0], C[1], h.tau * h.opts.sw_g);
    EO_CUDA_TRY(cudaGetLastError());
  }
  if ((rc = h.trace_end(TR_POST, st))) return rc;
  return EO_OK;
}

// One application of sum_p c_p (tau L - alpha_p)^{-1} restricted to poles
// [p0, p0 + np) with accumulation weights wgt (device [P][K]) and post constants C.
eo_status run_step(Handle& h, const double* uin, double* uout, int R, int p0, int np, const cd* wgt,
                   const double* C, cudaStream_t st) {
  Sweep s;
  eo_status rc = sweep_to_edges(h, uin, R, p0, np, wgt, s, st);
  if (rc) return rc;
  return finish_step(h, s, uin, uout, C, st);
}

}  // namespace

eo_status Handle::trace_begin(cudaStream_t st) {
  if (!timing) return EO_OK;
  if ((size_t)(2 * ev_used + 2) > ev_pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      EO_CUDA_TRY(cudaEventCreate(&e));
      ev_pool.push_back(e);
    }
  }
  EO_CUDA_TRY(cudaEventRecord(ev_pool[2 * ev_used], st));
  return EO_OK;
}

eo_status Handle::trace_end(int cls, cudaStream_t st) {
  if (!timing) return EO_OK;
  EO_CUDA_TRY(cudaEventRecord(ev_pool[2 * ev_used + 1], st));
  if ((int)ev_class.size() <= ev_used) ev_class.resize(ev_used + 1);
  ev_class[ev_used++] = cls;
  return EO_OK;
}

// Launch-shape autotuner.  For every merge level (both sweeps) and the root wall
// solve it times each candidate shape -- columns per block (1, 2, 4, 8) times
// k groups per row pass -- on the handle's own operators and workspace (three
// timed launches after one warm-up, CUDA events on the stream) and keeps the
// fastest.  It runs once per handle and n_rhs, before the first step; what it
// leaves in the workspace is overwritten by that step.
eo_status autotune(Handle& h, int R, cudaStream_t st) {
  if (h.tuned_R == R || !h.opts.autotune) return EO_OK;
  cudaStreamCaptureStatus cs;
  EO_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return EO_OK;   // keep the defaults inside a capture
  struct Ev {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Ev() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
  } ev;
  EO_CUDA_TRY(cudaEventCreate(&ev.a));
  EO_CUDA_TRY(cudaEventCreate(&ev.b));
  Sweep s = base_sweep(h, R, 0, h.P, h.wgt);
  const int L = h.plan.L();
  // time one launch function; returns ms per launch or a negative value on error
  auto timeit = [&](auto&& launch) -> float {
    if (launch()) return -1.f;
    if (cudaEventRecord(ev.a, st) != cudaSuccess) return -1.f;
    for (int i = 0; i < 3; ++i)
      if (launch()) return -1.f;
    if (cudaEventRecord(ev.b, st) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess) return -1.f;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) return -1.f;
    return ms / 3.f;
  };
  auto nc_list = [&](int nbox, int k, int rows) {
    std::vector<int> v;
    for (int nc = 1; nc <= 8; nc *= 2) {
      if (h.shared ? (nc > 1 && (long long)nbox * R < nc) : (R % nc != 0)) continue;
      if ((size_t)nc * (k + rows + 256) * sizeof(cd) > 200 * 1024) continue;
      v.push_back(nc);
    }
    return v;
  };
  auto nt_list = [&](int rows) {
    std::vector<int> v;
    const int rp = cmv_rp(rows);
    for (int ks = 1; ks <= 16 && rp * ks <= 256; ks *= 2) v.push_back(rp * ks);
    return v;
  };
  for (int l = 1; l <= L; ++l) {
    MergeArgs m = merge_args(h, l);
    LevelDev& ld = h.lv[l];
    float best = 1e30f;
    for (int nc : nc_list(m.nbox, m.n3, m.zu_rows))
      for (int nt : nt_list(m.sym ? m.rh : m.zu_rows)) {
        const int fmt = up_format(h, l, fused_plan(h, R).Lf);
        const float t = timeit([&] { return dispatch<UpMerge>(ld.fp32, nc, s, m, h.hA, h.hB, nt, fmt, st); });
        if (t < 0) return fail(EO_ERR_CUDA, "autotune: merge launch failed");
        if (t < best) { best = t; ld.up = Tuned{nc, nt}; }
      }
    if (!m.S) continue;
    best = 1e30f;
    for (int nc : nc_list(m.nbox, m.nbd, m.n3))
      for (int nt : nt_list(m.sym && m.Ss ? m.n3h : m.n3)) {
        const float t = timeit([&] { return dispatch<DownMerge>(ld.fp32, nc, s, m, h.E, nt, st); });
        if (t < 0) return fail(EO_ERR_CUDA, "autotune: merge launch failed");
        if (t < best) { best = t; ld.down = Tuned{nc, nt}; }
      }
  }
  if (h.fd) {
    const int nleaf = h.g.nlx * h.g.nly;
    float bu = 1e30f, bd = 1e30f;
    for (int nc : fd_ncol_candidates(h)) {
      float t = timeit([&] { return fd_up_kernel(h, s, nleaf, h.hA, nc, st); });
      if (t < 0) return fail(EO_ERR_CUDA, "autotune: leaf launch failed");
      if (t < bu) { bu = t; h.fd_ncol_up = nc; }
      int nchunk = 0;
      t = timeit([&] { return fd_down_leaf(h, s, nleaf, nc, nchunk, st); });
      if (t < 0) return fail(EO_ERR_CUDA, "autotune: leaf launch failed");
      if (t < bd) { bd = t; h.fd_ncol_down = nc; }
    }
  }
  if (h.g.periodic) {
    const Level& rl = h.plan.lv[L];
    RootArgs ra{rl.nbd, h.g.q, rl.sx * h.g.q, rl.sy * h.g.q, h.lv[L].bseg, h.aBinv, nullptr, nullptr, h.ustate, h.F};
    const int m = rl.nbd / 2;
    float best = 1e30f;
    for (int nc = 1; nc <= 8 && nc <= R; nc *= 2)
      for (int rs = 1; rs <= 4; rs *= 2)
        for (int nt : nt_list((m + rs - 1) / rs)) {
          if ((size_t)nc * (2 * m + 256) * sizeof(cd) > 200 * 1024) continue;
          const float t = timeit([&] { return dispatch<RootPer>(h.root_fp32, nc, s, ra, h.hA, h.E, nt, rs, st); });
          if (t < 0) return fail(EO_ERR_CUDA, "autotune: root launch failed");
          if (t < best) { best = t; h.root_tuned = Tuned{nc, nt, rs}; }
        }
  } else if (h.kind == EO_SW_WALLS) {
    const Level& rl = h.plan.lv[L];
    RootArgs ra{rl.nbd, h.g.q, rl.sx * h.g.q, rl.sy * h.g.q, h.lv[L].bseg, h.aBinv, h.bcoef, h.nu, h.ustate, 3,
                h.c4, h.c4idx, h.c4inv};
    float best = 1e30f;
    for (int nc = 1; nc <= 8 && nc <= R; nc *= 2)
      for (int rs = 1; rs <= (h.c4 ? 1 : 4); rs *= 2)
        for (int nt : nt_list(h.c4 ? h.c4 : (rl.nbd + rs - 1) / rs)) {
          if ((size_t)nc * (2 * rl.nbd + 256) * sizeof(cd) > 200 * 1024) continue;
          const float t = timeit([&] { return dispatch<RootSW>(h.root_fp32, nc, s, ra, h.hA, h.E, nt, rs, st); });
          if (t < 0) return fail(EO_ERR_CUDA, "autotune: root launch failed");
          if (t < best) { best = t; h.root_tuned = Tuned{nc, nt, rs}; }
        }
  }
  h.tuned_R = R;
  return EO_OK;
}

eo_status apply(Handle& h, double* u, int n_rhs, int n_steps, cudaStream_t st) {
  if (!u) return fail(EO_ERR_INVALID_ARG, "null state");
  if (n_rhs < 1 || n_rhs > h.R) return fail(EO_ERR_INVALID_ARG, "n_rhs out of range [1, max_rhs]");
  if (n_steps < 0) return fail(EO_ERR_INVALID_ARG, "negative n_steps");
  eo_status rc0 = autotune(h, n_rhs, st);
  if (rc0) return rc0;
  double* cur = u;
  double* nxt = h.ustate;
  eo_status rc;
  // Two or more steps and no tracing: record a pair of steps (u -> work -> u)
  // once as a CUDA graph for this (state, n_rhs) and replay it; the launch
  // sequence of a step is fixed, so the graph stays valid until the state
  // pointer or n_rhs changes.
  if (n_steps >= 2 && !h.timing && h.opts.use_graphs) {
    if (!h.graph_exec || h.graph_u != u || h.graph_R != n_rhs) {
      if (h.graph_exec) { cudaGraphExecDestroy(h.graph_exec); h.graph_exec = nullptr; }
      // record on a private stream (the legacy default stream cannot be
      // captured); the graph is then launched on the caller's stream
      if (!h.cap_st) EO_CUDA_TRY(cudaStreamCreateWithFlags(&h.cap_st, cudaStreamNonBlocking));
      cudaGraph_t graph;
      EO_CUDA_TRY(cudaStreamBeginCapture(h.cap_st, cudaStreamCaptureModeThreadLocal));
      eo_status rc1 = run_step(h, u, h.ustate, n_rhs, 0, h.P, h.wgt, h.C, h.cap_st);
      eo_status rc2 = rc1 ? rc1 : run_step(h, h.ustate, u, n_rhs, 0, h.P, h.wgt, h.C, h.cap_st);
      cudaError_t e = cudaStreamEndCapture(h.cap_st, &graph);
      if (rc2) return rc2;
      if (e != cudaSuccess) return fail(EO_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&h.graph_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(EO_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      h.graph_u = u;
      h.graph_R = n_rhs;
    }
    for (int i = 0; i + 1 < n_steps; i += 2) EO_CUDA_TRY(cudaGraphLaunch(h.graph_exec, st));
    if (n_steps % 2 == 0) return EO_OK;
    n_steps = 1;   // one more plain step below
  }
  for (int i = 0; i < n_steps; ++i) {
    if ((rc = run_step(h, cur, nxt, n_rhs, 0, h.P, h.wgt, h.C, st))) return rc;
    std::swap(cur, nxt);
  }
  if (cur != u)
    EO_CUDA_TRY(cudaMemcpyAsync(u, cur, sizeof(double) * (size_t)n_rhs * h.F * h.g.n_nodes,
                                cudaMemcpyDeviceToDevice, st));
  return EO_OK;
}

// out[k] = f_k(tau L) u for n_out pole-weight sets that share the poles (dense
// output, phi-functions): one pre-map, upward sweep, root and downward merge pass,
// then leaf interiors, pole sums and post-map once per set.
eo_status apply_functions(Handle& h, int n_out, const cd* wgts, const double* Cs, const double* u, double* out,
                          cudaStream_t st) {
  eo_status rc = autotune(h, 1, st);
  if (rc) return rc;
  Sweep s;
  if ((rc = sweep_to_edges(h, u, 1, 0, h.P, wgts, s, st))) return rc;
  const size_t nst = (size_t)h.F * h.g.n_nodes;
  for (int k = 0; k < n_out; ++k) {
    s.wgt = wgts + (size_t)k * h.P * h.K;
    if ((rc = finish_step(h, s, u, out + k * nst, Cs + 4 * k, st))) return rc;
  }
  return EO_OK;
}

// ---------------------------------------------------------------- the filter S(k0 Delta)
// Field column c of u ([ncol][n_nodes]) into the shallow-water state c of st ([c][3][n]):
// velocities zero, h = the field.
__global__ void k_filter_stage(const double* __restrict__ u, int ncol, long long n, double* __restrict__ st) {
  const long long tot = (long long)ncol * 3 * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / (3 * n), rem = i - c * 3 * n;
    st[i] = rem < 2 * n ? 0.0 : u[c * n + (rem - 2 * n)];
  }
}

// h of state c of st back into field column c of u.
__global__ void k_filter_unstage(const double* __restrict__ st, int ncol, long long n, double* __restrict__ u) {
  const long long tot = (long long)ncol * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / n, k = i - c * n;
    u[i] = st[(c * 3 + 2) * n + k];
  }
}

// S(k0 Delta) on ncol real fields, in place (Section 3.3).  The handle is a
// shallow-water handle with f = 0: its per-pole elliptic solve is
// (tau^2 g H Delta - alpha^2) w = alpha r for the state (0, 0, r), so the h field of
// the pole sum with the filter's weights is sum_m s_m alpha_m (k0 Delta - alpha_m^2)^{-1} r
// with k0 = tau^2 g H, the natural (Neumann) condition on walls.  Columns go through
// in groups of at most max_rhs, staged in two handle buffers.
eo_status apply_laplacian_filter(Handle& h, const cd* wgts, const double* C, double* u, int ncol,
                                 cudaStream_t st) {
  const long long n = h.g.n_nodes;
  const size_t per = (size_t)h.R * 3 * n;
  eo_status rc;
  if (!h.fstage && (rc = h.alloc((void**)&h.fstage, sizeof(double) * 2 * per, false))) return rc;
  double* in = h.fstage;
  double* out = h.fstage + per;
  for (int c0 = 0; c0 < ncol; c0 += h.R) {
    const int c = std::min(h.R, ncol - c0);
    const unsigned nb = (unsigned)std::min<long long>(4096, ((long long)c * 3 * n + 255) / 256);
    k_filter_stage<<<nb, 256, 0, st>>>(u + (size_t)c0 * n, c, n, in);
    EO_CUDA_TRY(cudaGetLastError());
    if ((rc = autotune(h, c, st))) return rc;
    Sweep s;
    if ((rc = sweep_to_edges(h, in, c, 0, h.P, wgts, s, st))) return rc;
    if ((rc = finish_step(h, s, in, out, C, st))) return rc;
    k_filter_unstage<<<nb, 256, 0, st>>>(out, c, n, u + (size_t)c0 * n);
    EO_CUDA_TRY(cudaGetLastError());
  }
  return EO_OK;
}

// ---------------------------------------------------------------- batches of instances
Batch::~Batch() {
  if (exec) cudaGraphExecDestroy(exec);
  for (cudaStream_t s : st) cudaStreamDestroy(s);
  if (st0) cudaStreamDestroy(st0);
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
}

// Record one step pair of every instance (u -> workspace -> u) as parallel
// branches of one CUDA graph: a fork event on a private stream, one branch
// stream per instance, join events back.  Launch shapes are tuned first,
// outside the capture.
eo_status batch_build(Batch& b) {
  const int n = (int)b.h.size();
  for (int i = 0; i < n; ++i) {
    eo_status rc = autotune(*b.h[i], b.R[i], nullptr);
    if (rc) return rc;
  }
  EO_CUDA_TRY(cudaStreamCreateWithFlags(&b.st0, cudaStreamNonBlocking));
  b.st.assign(n, nullptr);
  for (int i = 0; i < n; ++i) EO_CUDA_TRY(cudaStreamCreateWithFlags(&b.st[i], cudaStreamNonBlocking));
  b.ev.assign(n + 1, nullptr);
  for (int i = 0; i <= n; ++i) EO_CUDA_TRY(cudaEventCreateWithFlags(&b.ev[i], cudaEventDisableTiming));
  EO_CUDA_TRY(cudaDeviceSynchronize());
  EO_CUDA_TRY(cudaStreamBeginCapture(b.st0, cudaStreamCaptureModeThreadLocal));
  eo_status rc = EO_OK;
  cudaError_t e = cudaEventRecord(b.ev[n], b.st0);
  for (int i = 0; i < n && !rc && e == cudaSuccess; ++i) {
    Handle& h = *b.h[i];
    e = cudaStreamWaitEvent(b.st[i], b.ev[n], 0);
    if (e != cudaSuccess) break;
    rc = run_step(h, b.u[i], h.ustate, b.R[i], 0, h.P, h.wgt, h.C, b.st[i]);
    if (!rc) rc = run_step(h, h.ustate, b.u[i], b.R[i], 0, h.P, h.wgt, h.C, b.st[i]);
    if (!rc) e = cudaEventRecord(b.ev[i], b.st[i]);
    if (!rc && e == cudaSuccess) e = cudaStreamWaitEvent(b.st0, b.ev[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b.st0, &graph);
  if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
  if (e != cudaSuccess || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(EO_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : ec));
  }
  e = cudaGraphInstantiate(&b.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(EO_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
  return EO_OK;
}

eo_status batch_apply(Batch& b, int n_steps, cudaStream_t st) {
  if (n_steps < 0) return fail(EO_ERR_INVALID_ARG, "negative n_steps");
  for (int i = 0; i + 1 < n_steps; i += 2) EO_CUDA_TRY(cudaGraphLaunch(b.exec, st));
  if (n_steps % 2) {
    for (size_t i = 0; i < b.h.size(); ++i) {
      eo_status rc = apply(*b.h[i], b.u[i], b.R[i], 1, st);
      if (rc) return rc;
    }
  }
  return EO_OK;
}

// Weights of the two runs of one resolvent: pole j alone with weight c = 1 (real
// part) or c = -i (imaginary part); w[k] are the K accumulation weights of that
// pole and C the post-map constants.
static void resolvent_weights(const Handle& h, int j, std::complex<double> c, cd w[3], double C[4]) {
  const std::complex<double> al = h.alpha[j];
  for (int k = 0; k < 3; ++k) w[k] = make_double2(0.0, 0.0);
  for (int k = 0; k < 4; ++k) C[k] = 0.0;
  if (h.kind == EO_WAVE_DIRICHLET) {
    const std::complex<double> w0 = c, w1 = c * h.tau / al;
    w[0] = make_double2(w0.real(), w0.imag());
    w[1] = make_double2(w1.real(), w1.imag());
    C[0] = (c / al).real();
  } else {
    const double tf = h.tau * h.opts.sw_f;
    const std::complex<double> D = al * al + tf * tf;
    const std::complex<double> w0 = c, w1 = c * (-al / D), w2 = c * (-tf / D);
    w[0] = make_double2(w0.real(), w0.imag());
    w[1] = make_double2(w1.real(), w1.imag());
    w[2] = make_double2(w2.real(), w2.imag());
    C[0] = w1.real();
    C[1] = w2.real();
  }
}

// x = (tau L - alpha_j)^{-1} u: the pole-sum pipeline run for pole j alone with
// weight 1 (real part) and weight -i (imaginary part); every post-map is linear
// with real coefficients in (weight * solution), so the two runs give Re and Im.
// The two scratch buffers are stream-ordered allocations, released on every exit.
eo_status apply_resolvent(Handle& h, int j, const double* u, double* x, cudaStream_t st) {
  if (j < 0 || j >= h.P) return fail(EO_ERR_INVALID_ARG, "pole index out of range");
  const std::complex<double> ws[2] = {1.0, std::complex<double>(0.0, -1.0)};
  const size_t nst = (size_t)h.F * h.g.n_nodes;
  struct Scratch {
    cudaStream_t st;
    void* p[2] = {nullptr, nullptr};
    ~Scratch() { for (void* v : p) if (v) cudaFreeAsync(v, st); }
  } sc{st};
  EO_CUDA_TRY(cudaMallocAsync(&sc.p[0], sizeof(cd) * h.P * h.K, st));
  EO_CUDA_TRY(cudaMallocAsync(&sc.p[1], sizeof(double) * nst * 2, st));
  cd* tmpw = (cd*)sc.p[0];
  double* outb = (double*)sc.p[1];
  // one host table per part (the copies are stream-ordered behind the kernels that
  // read the previous table; the host tables live until the final synchronisation)
  std::vector<cd> w(2 * (size_t)h.P * h.K, make_double2(0.0, 0.0));
  for (int part = 0; part < 2; ++part) {
    cd wj[3];
    double C[4];
    resolvent_weights(h, j, ws[part], wj, C);
    cd* wp = w.data() + (size_t)part * h.P * h.K;
    for (int k = 0; k < h.K; ++k) wp[(size_t)j * h.K + k] = wj[k];
    EO_CUDA_TRY(cudaMemcpyAsync(tmpw, wp, sizeof(cd) * h.P * h.K, cudaMemcpyHostToDevice, st));
    eo_status rc = run_step(h, u, outb + part * nst, 1, j, 1, (const cd*)tmpw, C, st);
    if (rc) {
      cudaStreamSynchronize(st);
      return rc;
    }
  }
  // interleave (re, im)
  EO_CUDA_TRY(cudaMemcpy2DAsync(x, 2 * sizeof(double), outb, sizeof(double), sizeof(double), nst,
                                cudaMemcpyDeviceToDevice, st));
  EO_CUDA_TRY(cudaMemcpy2DAsync(x + 1, 2 * sizeof(double), outb + nst, sizeof(double), sizeof(double), nst,
                                cudaMemcpyDeviceToDevice, st));
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  return EO_OK;
}

// ---------------------------------------------------------------- resolvent without allocation
// Some callers cannot allocate device memory at the moment they call: host
// threads that must stay off the device allocator (it takes locks and can
// synchronise the device), and embedders that hand every byte of the GPU to their
// own memory pool, where any outside cudaMalloc fails.  eo_apply_resolvent takes
// two scratch buffers from cudaMallocAsync on every call; this variant takes them
// from a fixed file-scope device array instead and allocates nothing.
//
// The array is kNoAllocDoubles doubles (16 MiB); every GPU that loads the library
// holds it until the process exits.  It holds the selected pole's K accumulation
// weights (kNoAllocWeights doubles) and the real and imaginary outputs
// (2 x fields x nodes doubles); larger problems are rejected with
// EO_ERR_INVALID_ARG.  All calls share the array and each keeps what the previous
// call left there (the weights are rewritten on the device by every call), so
// calls whose work overlaps on the GPU (different streams, or different handles
// on one device without ordering) race on it.
static constexpr size_t kNoAllocDoubles = 2u << 20;
static constexpr size_t kNoAllocWeights = 16;   // >= 2 * K doubles, keeps the outputs 128-byte aligned
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// w[k] of the selected pole into the scratch row (one thread per weight)
__global__ void k_set_weights(cd* __restrict__ dst, int K, cd w0, cd w1, cd w2) {
  const int k = threadIdx.x;
  if (k < K) dst[k] = k == 0 ? w0 : (k == 1 ? w1 : w2);
}

namespace {
std::mutex g_noalloc_mu;
std::vector<double*> g_noalloc_ptr;   // per device ordinal; null until set up

// Device address of the scratch array on the current device.  The first call
// on a device looks it up with that device current; later calls reuse it.
eo_status noalloc_scratch(double** out) {
  int dev = 0;
  EO_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if ((int)g_noalloc_ptr.size() <= dev) g_noalloc_ptr.resize(dev + 1, nullptr);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(EO_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return EO_OK;
}
}  // namespace

eo_status apply_resolvent_noalloc(Handle& h, int j, const double* u, double* x, cudaStream_t st) {
  if (j < 0 || j >= h.P) return fail(EO_ERR_INVALID_ARG, "pole index out of range");
  const size_t nst = (size_t)h.F * h.g.n_nodes;
  if (kNoAllocWeights + 2 * nst > kNoAllocDoubles)
    return fail(EO_ERR_INVALID_ARG, "problem too large for the no-allocation scratch (" +
                                        std::to_string(kNoAllocWeights + 2 * nst) + " doubles needed, " +
                                        std::to_string(kNoAllocDoubles) + " available)");
  double* scratch = nullptr;
  eo_status rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cd* wrow = (cd*)scratch;                     // the K weights of pole j
  double* outb = scratch + kNoAllocWeights;    // Re part, then Im part
  // The kernels read the weight of pole p at wgt[p * K + k], here only for p = j:
  // offset the table so that row j is the scratch row.
  const cd* wtab = wrow - (ptrdiff_t)j * h.K;
  const std::complex<double> ws[2] = {1.0, std::complex<double>(0.0, -1.0)};
  for (int part = 0; part < 2; ++part) {
    cd w[3];
    double C[4];
    resolvent_weights(h, j, ws[part], w, C);
    k_set_weights<<<1, 32, 0, st>>>(wrow, h.K, w[0], w[1], w[2]);
    EO_CUDA_TRY(cudaGetLastError());
    if ((rc = run_step(h, u, outb + part * nst, 1, j, 1, wtab, C, st))) return rc;
  }
  EO_CUDA_TRY(cudaMemcpy2DAsync(x, 2 * sizeof(double), outb, sizeof(double), sizeof(double), nst,
                                cudaMemcpyDeviceToDevice, st));
  EO_CUDA_TRY(cudaMemcpy2DAsync(x + 1, 2 * sizeof(double), outb + nst, sizeof(double), sizeof(double), nst,
                                cudaMemcpyDeviceToDevice, st));
  return EO_OK;
}

int fused_levels(const Handle& h, int R) { return fused_plan(h, R).Lf; }

}  // namespace eo
