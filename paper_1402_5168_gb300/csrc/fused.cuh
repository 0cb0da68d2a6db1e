// The low merge levels of both sweeps in one launch each (reflection-symmetric
// levels of shared per-level operators, the even/odd blocks of the merge kernels in
// apply.cu).  A block owns one pole and one box of level Lf (a subtree of 2^Lf leaves)
// and runs levels 1 .. Lf of it with 256 threads and up to 8 columns per block
// product, instead of one launch per level with one- and two-warp blocks.
//   up:   the boundary data of levels 1 .. Lf-1 stay in shared memory; level Lf goes
//         to the global workspace (the buffer the next level reads), and every level's
//         interface corrections w3 go to their global arrays as in the per-level kernels;
//   down: interface values are written to and read from the global edge array E, whose
//         entries inside the subtree belong to this block alone.
// The arithmetic per column is that of k_up_merge_sym / k_down_merge_sym.
#pragma once

#include "sweep.cuh"

namespace eo {

constexpr int FUSED_MAX = 4;   // levels fused at most (subtrees of up to 16 leaves)

struct FusedLevels {
  int Lf = 0;                       // levels 1 .. Lf are fused
  int nbx[FUSED_MAX + 1], nby[FUSED_MAX + 1];   // boxes per row / column, levels 0 .. Lf
  MergeArgs m[FUSED_MAX + 1];       // levels 1 .. Lf
  int hs = 0;                       // cd entries of one shared boundary buffer
};

// box (global index at level l) of local box lb in subtree (SX, SY) of level Lf
__device__ __forceinline__ int fused_box(const FusedLevels& f, int l, int SX, int SY, int lb) {
  const int fx = f.nbx[l] / f.nbx[f.Lf], fy = f.nby[l] / f.nby[f.Lf];
  return (SY * fy + lb / fx) * f.nbx[l] + SX * fx + lb % fx;
}
// local index in subtree (SX, SY) of global box b of level l
__device__ __forceinline__ int fused_local(const FusedLevels& f, int l, int SX, int SY, int b) {
  const int fx = f.nbx[l] / f.nbx[f.Lf], fy = f.nby[l] / f.nby[f.Lf];
  const int bx = b % f.nbx[l], by = b / f.nbx[l];
  return (by - SY * fy) * fx + (bx - SX * fx);
}
__device__ __forceinline__ int fused_nloc(const FusedLevels& f, int l) {
  return (f.nbx[l] / f.nbx[f.Lf]) * (f.nby[l] / f.nby[f.Lf]);
}

// One group of NC columns (c0 ..) of up level l.  Column c = lb * R + r.
template <int NC, typename TA>
__device__ void fused_up_group(const Sweep& s, const FusedLevels& f, int l, int SX, int SY, int pl, int c0,
                               const cd* __restrict__ h0, const cd* Hin, cd* Hout, cd* __restrict__ hout_g,
                               TA* Bs, cd* Cs, cd* red) {
  const MergeArgs& m = f.m[l];
  const int p = s.p0 + pl, R = s.R;
  const int n3 = m.n3, n3h = m.n3h, rh = m.rh;
  const int nloc = fused_nloc(f, l), nlocc = fused_nloc(f, l - 1);
  const int ncols = nloc * R;
  // boundary value k of child box cb (global, level l-1) for right-hand side r
  auto hin = [&](int cb, int r, int k) -> cd {
    if (l == 1) return h0[(((long long)pl * R + r) * m.nbox_c + cb) * m.nbd_c + k];
    return Hin[((long long)r * nlocc + fused_local(f, l - 1, SX, SY, cb)) * m.nbd_c + k];
  };
  for (int e = threadIdx.x; e < NC * n3h; e += blockDim.x) {
    const int c = e / n3h, t = e - c * n3h;
    cd ev = make_double2(0.0, 0.0), od = make_double2(0.0, 0.0);
    if (c0 + c < ncols) {
      const int lb = (c0 + c) / R, r = (c0 + c) - lb * R;
      int ca, cb;
      children(m, fused_box(f, l, SX, SY, lb), ca, cb);
      const int tj = n3 - 1 - t;
      const cd x1 = hin(ca, r, m.a3[t]), y1 = hin(cb, r, m.b3[t]);
      const cd x2 = hin(ca, r, m.a3[tj]), y2 = hin(cb, r, m.b3[tj]);
      const double ar = x1.x + y1.x, ai = x1.y + y1.y, br = x2.x + y2.x, bi = x2.y + y2.y;
      ev = make_double2(0.5 * (ar + br), 0.5 * (ai + bi));
      od = make_double2(0.5 * (ar - br), 0.5 * (ai - bi));
    }
    Bs[c * n3 + t] = Cv<TA>::from(ev);
    Bs[c * n3 + n3h + t] = Cv<TA>::from(od);
  }
  __syncthreads();
  const TA* A = (const TA*)m.ZUs + (long long)p * m.zsps;
  cmv<NC, TA>(A, rh, rh, n3h, Bs, n3, Cs, red);
  cmv<NC, TA>(A + (long long)rh * n3h, rh, rh, n3h, Bs + n3h, n3, Cs + (size_t)NC * rh, red);
  const cd* Ce = Cs;
  const cd* Co = Cs + (size_t)NC * rh;
  for (int e = threadIdx.x; e < NC * m.zu_rows; e += blockDim.x) {
    const int c = e / m.zu_rows, row = e - c * m.zu_rows;
    if (c0 + c >= ncols) continue;
    const int lb = (c0 + c) / R, r = (c0 + c) - lb * R;
    const int box = fused_box(f, l, SX, SY, lb);
    if (row < n3) {
      const int sr = row < n3h ? row : n3 - 1 - row;
      const double sg = row < n3h ? 1.0 : -1.0;
      const cd a = Ce[c * rh + sr], b = Co[c * rh + sr];
      m.w3[(((long long)pl * R + r) * m.nbox + box) * n3 + row] = make_double2(a.x + sg * b.x, a.y + sg * b.y);
    } else {
      const int i = row - n3;
      const int k = n3h + m.orb[i];
      const double sg = (double)m.osg[i];
      const cd a = Ce[c * rh + k], b = Co[c * rh + k];
      int ca, cb;
      children(m, box, ca, cb);
      const cd x = hin(m.par_child[i] ? cb : ca, r, m.par_idx[i]);
      const cd v = make_double2(x.x + a.x + sg * b.x, x.y + a.y + sg * b.y);
      if (l == f.Lf) hout_g[(((long long)pl * R + r) * m.nbox + box) * m.nbd + i] = v;
      else Hout[((long long)r * nloc + lb) * m.nbd + i] = v;
    }
  }
  __syncthreads();
}

// Grid (level-Lf boxes, poles in this call), 256 threads.  Shared memory: two
// boundary buffers of f.hs entries, then the block-product scratch (8 columns).
template <typename TA>
__global__ void __launch_bounds__(256) k_up_fused(Sweep s, FusedLevels f, const cd* __restrict__ h0,
                                                  cd* __restrict__ hout) {
  extern __shared__ cd fsm[];
  const int sub = blockIdx.x, pl = blockIdx.y;
  const int SX = sub % f.nbx[f.Lf], SY = sub / f.nbx[f.Lf];
  cd* H0 = fsm;
  cd* H1 = fsm + f.hs;
  int n3max = 0, rhmax = 0;
  for (int l = 1; l <= f.Lf; ++l) {
    n3max = max(n3max, f.m[l].n3);
    rhmax = max(rhmax, f.m[l].rh);
  }
  TA* Bs = (TA*)(fsm + 2 * f.hs);
  cd* Cs = after(Bs, (size_t)8 * n3max);
  cd* red = Cs + 2 * 8 * rhmax;
  for (int l = 1; l <= f.Lf; ++l) {
    const cd* Hin = (l % 2 == 0) ? H1 : H0;   // level l-1's buffer (l - 1 odd: H1)
    cd* Hout = (l % 2 == 0) ? H0 : H1;
    const int ncols = fused_nloc(f, l) * s.R;
    for (int c0 = 0; c0 < ncols;) {
      const int rem = ncols - c0;
      if (rem >= 8) { fused_up_group<8, TA>(s, f, l, SX, SY, pl, c0, h0, Hin, Hout, hout, Bs, Cs, red); c0 += 8; }
      else if (rem >= 4) { fused_up_group<4, TA>(s, f, l, SX, SY, pl, c0, h0, Hin, Hout, hout, Bs, Cs, red); c0 += 4; }
      else if (rem >= 2) { fused_up_group<2, TA>(s, f, l, SX, SY, pl, c0, h0, Hin, Hout, hout, Bs, Cs, red); c0 += 2; }
      else { fused_up_group<1, TA>(s, f, l, SX, SY, pl, c0, h0, Hin, Hout, hout, Bs, Cs, red); c0 += 1; }
    }
  }
}

// One group of NC columns (c0 ..) of down level l: the parent boundary values enter
// only through their orbit sums a_r, b_r (k_down_merge_sym); u3 goes to E.
template <int NC, typename TA>
__device__ void fused_down_group(const Sweep& s, const FusedLevels& f, int l, int SX, int SY, int pl, int c0,
                                 cd* __restrict__ E, TA* Bs, cd* Cs, cd* red) {
  const MergeArgs& m = f.m[l];
  const int p = s.p0 + pl, R = s.R, q = s.q;
  const int n3 = m.n3, n3h = m.n3h, nbq = m.nbq;
  const int ncols = fused_nloc(f, l) * R;
  for (int e = threadIdx.x; e < NC * nbq; e += blockDim.x) {
    const int c = e / nbq, rr = e - c * nbq;
    cd a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    if (c0 + c < ncols) {
      const int lb = (c0 + c) / R, r = (c0 + c) - lb * R;
      const int box = fused_box(f, l, SX, SY, lb);
      const cd* Er = E + ((long long)pl * R + r) * s.n_edge;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int i = m.mem[4 * rr + g];
        const cd v = Er[(long long)m.bseg[box * m.nseg + i / q] * q + (i % q)];
        const double sg = g < 2 ? 1.0 : -1.0;
        a.x += v.x; a.y += v.y;
        b.x += sg * v.x; b.y += sg * v.y;
      }
    }
    Bs[c * 2 * nbq + rr] = Cv<TA>::from(a);
    Bs[c * 2 * nbq + nbq + rr] = Cv<TA>::from(b);
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
    const int lb = (c0 + c) / R, r = (c0 + c) - lb * R;
    const int box = fused_box(f, l, SX, SY, lb);
    const int sr = row < n3h ? row : n3 - 1 - row;
    const double sg = row < n3h ? 1.0 : -1.0;
    const cd a = Ce[c * n3h + sr], b = Co[c * n3h + sr];
    const cd w = m.w3[(((long long)pl * R + r) * m.nbox + box) * n3 + row];
    E[((long long)pl * R + r) * s.n_edge + (long long)m.iseg[box * n3s + row / q] * q + (row % q)] =
        make_double2(w.x + a.x + sg * b.x, w.y + a.y + sg * b.y);
  }
  __syncthreads();   // this level's interface values are the next level's boundary data
}

template <typename TA>
__global__ void __launch_bounds__(256) k_down_fused(Sweep s, FusedLevels f, cd* __restrict__ E) {
  extern __shared__ cd fsm[];
  const int sub = blockIdx.x, pl = blockIdx.y;
  const int SX = sub % f.nbx[f.Lf], SY = sub / f.nbx[f.Lf];
  int kmax = 0, n3max = 0;
  for (int l = 1; l <= f.Lf; ++l) {
    kmax = max(kmax, 2 * f.m[l].nbq);
    n3max = max(n3max, f.m[l].n3);
  }
  TA* Bs = (TA*)fsm;
  cd* Cs = after(Bs, (size_t)8 * kmax);
  cd* red = Cs + 8 * n3max;
  for (int l = f.Lf; l >= 1; --l) {
    const int ncols = fused_nloc(f, l) * s.R;
    for (int c0 = 0; c0 < ncols;) {
      const int rem = ncols - c0;
      if (rem >= 8) { fused_down_group<8, TA>(s, f, l, SX, SY, pl, c0, E, Bs, Cs, red); c0 += 8; }
      else if (rem >= 4) { fused_down_group<4, TA>(s, f, l, SX, SY, pl, c0, E, Bs, Cs, red); c0 += 4; }
      else if (rem >= 2) { fused_down_group<2, TA>(s, f, l, SX, SY, pl, c0, E, Bs, Cs, red); c0 += 2; }
      else { fused_down_group<1, TA>(s, f, l, SX, SY, pl, c0, E, Bs, Cs, red); c0 += 1; }
    }
  }
}

}  // namespace eo
