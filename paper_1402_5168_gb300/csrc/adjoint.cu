// Adjoint of the time step: y <- G^T y, G the real linear map of one step
// u -> Re sum_p c_p post_p(x_p), x_p = (tau L - alpha_p)^{-1} u (Section 1.1,
// eq. def_RM, with the conjugate-pole form of Section 3.3).
//
// With the bilinear pairing <a, b> = sum a_i b_i, a real seed y gives per pole the
// complex seed z_p = sum_k w_pk y_k on the elliptic solution (w_pk the pole-sum
// weights of the forward accumulation), and G^T y = Pre^T Re sum_p coef_pk
// Sol_p^T z_p + (direct terms of the post-map).  Sol_p^T, the plain transpose of
// the nested-dissection solve, runs the forward sweeps backwards with every
// stored block transposed and every gather turned into a scatter:
//   leaves down^T:  g_bar = X^T z_int,  e_bar(leaf edges) += Y^T z_int
//   merges down^T (levels 1..L): w3_bar = e_bar(interface),
//                   e_bar(parent boundary) += S^T e_bar(interface)
//   merges up^T (levels L..1): s3_bar = [-Z; U]^T [w3_bar; h_bar_parent],
//                   h_bar_alpha(3) = h_bar_beta(3) = s3_bar, exterior parts copied
//   leaves up^T:    g_bar += H^T h_bar_leaf
// Transposed block products read each column of a block with one warp
// (coalesced) and reduce across the warp.  Scatters onto edges shared by
// neighbouring boxes use FP64 atomic adds.
#include <algorithm>
#include <string>

#include "sweep.cuh"

namespace eo {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Out[c][j] = sum_{r<rows} A[r + j*lda] X[c][r] for j < k: one warp per column.
// Xs: shared [NC][xb] in TA; Out: shared [NC][k] (FP64).
template <int NC, typename TA>
__device__ void cmvT(const TA* __restrict__ A, int lda, int rows, int k, const TA* Xs, int xb, cd* Out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < k; j += nw) {
    typename Cv<TA>::Acc acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = Cv<TA>::zero();
    const TA* Aj = A + (size_t)j * lda;
    for (int r = lane; r < rows; r += 32) {
      const TA a = operator_ld(Aj + r);
#pragma unroll
      for (int c = 0; c < NC; ++c) Cv<TA>::mac(acc[c], a, Xs[c * xb + r]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      cd v = Cv<TA>::to(acc[c]);
      v.x = warp_sum(v.x);
      v.y = warp_sum(v.y);
      if (lane == 0) Out[c * k + j] = v;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void atomic_cadd(cd* p, cd v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// seed of pole p at a node from the real seed fields: z = sum_k w_pk y_k
__device__ __forceinline__ cd seed(const Sweep& s, int p, int r, long long node) {
  cd z = make_double2(0.0, 0.0);
  for (int kk = 0; kk < s.K; ++kk) {
    const double y = s.src[kk][r * s.src_rs[kk] + node];
    const cd w = s.wgt[p * s.K + kk];
    z.x += w.x * y;
    z.y += w.y * y;
  }
  return z;
}

// ---------------------------------------------------------------- leaves down^T
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_adj_down_leaf(Sweep s, const void* XYv, long long xps, long long xbs,
                                                       int nleaf, cd* __restrict__ gbar, cd* __restrict__ ybar) {
  extern __shared__ cd smem[];
  const TA* XY = (const TA*)XYv;
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int ni = s.ni, nb = s.nb, k = ni + nb;
  const int ncols = nleaf * s.R;
  const int c0 = blockIdx.x * NC;
  TA* Xs = (TA*)smem;
  cd* Out = after(Xs, (size_t)NC * ni);
  for (int e = threadIdx.x; e < NC * ni; e += blockDim.x) {
    const int c = e / ni, i = e - c * ni;
    cd z = make_double2(0.0, 0.0);
    if (c0 + c < ncols) {
      int box, r;
      col_box(c0 + c, s.R, box, r);
      z = seed(s, p, r, (long long)box * ni + i);
    }
    Xs[e] = Cv<TA>::from(z);
  }
  __syncthreads();
  int box0, r0;
  col_box(c0, s.R, box0, r0);
  cmvT<NC, TA>(XY + (long long)p * xps + (s.shared ? 0 : (long long)box0 * xbs), ni, ni, k, Xs, ni, Out);
  for (int e = threadIdx.x; e < NC * k; e += blockDim.x) {
    const int c = e / k, j = e - c * k;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    const long long base = ((long long)pl * s.R + r) * nleaf + box;
    if (j < ni) gbar[base * ni + j] = Out[e];
    else ybar[base * nb + (j - ni)] = Out[e];
  }
}

// e_bar on every edge node: seed there plus the Y^T contributions of the (one or
// two) leaves whose boundary contains the node, in a fixed order.
__global__ void k_adj_edges(Sweep s, int nlx, int nly, const cd* __restrict__ ybar, cd* __restrict__ E) {
  const long long tot = (long long)s.P * s.R * s.n_edge;
  const int q = s.q, nb = s.nb;
  const long long n_hseg = (long long)nlx * (nly + 1);
  const int nleaf = nlx * nly;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t % s.n_edge;
    const long long pr = t / s.n_edge;
    const int r = (int)(pr % s.R), pl = (int)(pr / s.R);
    const long long seg = e / q;
    const int o = (int)(e % q);
    cd v = seed(s, s.p0 + pl, r, s.n_int + e);
    int la = -1, pa = 0, lb = -1, pb = 0;   // leaves and boundary positions
    if (seg < n_hseg) {
      const int line = (int)(seg / nlx), a = (int)(seg % nlx);
      if (line > 0) { la = (line - 1) * nlx + a; pa = 2 * q + o; }     // N side of the leaf below
      if (line < nly) { lb = line * nlx + a; pb = o; }                 // S side of the leaf above
    } else {
      const long long sv = seg - n_hseg;
      const int b = (int)(sv / (nlx + 1)), line = (int)(sv % (nlx + 1));
      if (line > 0) { la = b * nlx + line - 1; pa = q + o; }           // E side of the left leaf
      if (line < nlx) { lb = b * nlx + line; pb = 3 * q + o; }         // W side of the right leaf
    }
    const long long base = ((long long)pl * s.R + r) * nleaf;
    if (la >= 0) { const cd y = ybar[(base + la) * nb + pa]; v.x += y.x; v.y += y.y; }
    if (lb >= 0) { const cd y = ybar[(base + lb) * nb + pb]; v.x += y.x; v.y += y.y; }
    E[t] = v;
  }
}

// ---------------------------------------------------------------- merges down^T
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_adj_down_merge(Sweep s, MergeArgs m, cd* __restrict__ E) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int ncols = m.nbox * s.R;
  const int c0 = blockIdx.x * NC;
  const int q = s.q, n3s = m.n3 / q;
  TA* Xs = (TA*)smem;
  cd* Out = after(Xs, (size_t)NC * m.n3);
  for (int e = threadIdx.x; e < NC * m.n3; e += blockDim.x) {
    const int c = e / m.n3, t = e - c * m.n3;
    cd v = make_double2(0.0, 0.0);
    if (c0 + c < ncols) {
      int box, r;
      col_box(c0 + c, s.R, box, r);
      v = E[((long long)pl * s.R + r) * s.n_edge + (long long)m.iseg[box * n3s + t / q] * q + (t % q)];
      m.w3[(((long long)pl * s.R + r) * m.nbox + box) * m.n3 + t] = v;
    }
    Xs[e] = Cv<TA>::from(v);
  }
  __syncthreads();
  if (!m.S) return;
  int box0, r0;
  col_box(c0, s.R, box0, r0);
  const TA* A = (const TA*)m.S + (long long)p * m.sps + (s.shared ? 0 : (long long)box0 * m.sbs);
  cmvT<NC, TA>(A, m.n3, m.n3, m.nbd, Xs, m.n3, Out);
  for (int e = threadIdx.x; e < NC * m.nbd; e += blockDim.x) {
    const int c = e / m.nbd, i = e - c * m.nbd;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    atomic_cadd(&E[((long long)pl * s.R + r) * s.n_edge + (long long)m.bseg[box * m.nseg + i / q] * q + (i % q)],
                Out[e]);
  }
}

// ---------------------------------------------------------------- merges up^T
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_adj_up_merge(Sweep s, MergeArgs m, const cd* __restrict__ hpar,
                                                      cd* __restrict__ hchild) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int ncols = m.nbox * s.R;
  const int c0 = blockIdx.x * NC;
  TA* Xs = (TA*)smem;
  cd* Out = after(Xs, (size_t)NC * m.zu_rows);
  for (int e = threadIdx.x; e < NC * m.zu_rows; e += blockDim.x) {
    const int c = e / m.zu_rows, row = e - c * m.zu_rows;
    cd v = make_double2(0.0, 0.0);
    if (c0 + c < ncols) {
      int box, r;
      col_box(c0 + c, s.R, box, r);
      if (row < m.n3) v = m.w3[(((long long)pl * s.R + r) * m.nbox + box) * m.n3 + row];
      else v = hpar[(((long long)pl * s.R + r) * m.nbox + box) * m.nbd + (row - m.n3)];
    }
    Xs[e] = Cv<TA>::from(v);
  }
  __syncthreads();
  int box0, r0;
  col_box(c0, s.R, box0, r0);
  const TA* A = (const TA*)m.ZU + (long long)p * m.zps + (s.shared ? 0 : (long long)box0 * m.zbs);
  cmvT<NC, TA>(A, m.zu_rows, m.zu_rows, m.n3, Xs, m.zu_rows, Out);
  // interface positions of both children get s3_bar; exterior positions copy h_bar_parent
  for (int e = threadIdx.x; e < NC * (m.n3 + m.nbd); e += blockDim.x) {
    const int c = e / (m.n3 + m.nbd), i = e - c * (m.n3 + m.nbd);
    if (c0 + c >= ncols) continue;
    int box, r, ca, cb;
    col_box(c0 + c, s.R, box, r);
    children(m, box, ca, cb);
    cd* hr = hchild + ((long long)pl * s.R + r) * m.nbox_c * m.nbd_c;
    if (i < m.n3) {
      const cd v = Out[c * m.n3 + i];
      hr[(long long)ca * m.nbd_c + m.a3[i]] = v;
      hr[(long long)cb * m.nbd_c + m.b3[i]] = v;
    } else {
      const int ip = i - m.n3;
      const bool has_par = m.zu_rows > m.n3;
      const cd v = has_par ? hpar[(((long long)pl * s.R + r) * m.nbox + box) * m.nbd + ip] : make_double2(0.0, 0.0);
      hr[(long long)(m.par_child[ip] ? cb : ca) * m.nbd_c + m.par_idx[ip]] = v;
    }
  }
}

// ---------------------------------------------------------------- leaves up^T + pole sums
// g_bar_total = g_bar + H^T h_bar_leaf;  acc_k += Re(coef_pk g_bar_total) over the
// block's poles; partials [chunk][rhs][K][n_int].
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_adj_up_leaf(Sweep s, const void* Hv, long long hps, long long hbs,
                                                     int nleaf, int ppc, const cd* __restrict__ h0,
                                                     const cd* __restrict__ gbar, double* __restrict__ part) {
  extern __shared__ cd smem[];
  const TA* H = (const TA*)Hv;
  const int ni = s.ni, nb = s.nb;
  const int ncols = nleaf * s.R;
  const int c0 = blockIdx.x * NC;
  const int chunk = blockIdx.y;
  TA* Xs = (TA*)smem;
  cd* Out = after(Xs, (size_t)NC * nb);
  double* acc = (double*)(Out + NC * ni);   // [NC][K][ni]
  for (int e = threadIdx.x; e < NC * s.K * ni; e += blockDim.x) acc[e] = 0.0;
  int box0, r0;
  col_box(c0, s.R, box0, r0);
  const int pbeg = chunk * ppc, pend = min(s.P, pbeg + ppc);
  for (int pl = pbeg; pl < pend; ++pl) {
    const int p = s.p0 + pl;
    __syncthreads();
    for (int e = threadIdx.x; e < NC * nb; e += blockDim.x) {
      const int c = e / nb, i = e - c * nb;
      cd v = make_double2(0.0, 0.0);
      if (c0 + c < ncols) {
        int box, r;
        col_box(c0 + c, s.R, box, r);
        v = h0[(((long long)pl * s.R + r) * nleaf + box) * nb + i];
      }
      Xs[e] = Cv<TA>::from(v);
    }
    __syncthreads();
    cmvT<NC, TA>(H + (long long)p * hps + (s.shared ? 0 : (long long)box0 * hbs), nb, nb, ni, Xs, nb, Out);
    cd cf[3];
    for (int kk = 0; kk < s.K; ++kk) cf[kk] = s.coef[p * s.K + kk];
    for (int e = threadIdx.x; e < NC * ni; e += blockDim.x) {
      const int c = e / ni, i = e - c * ni;
      if (c0 + c >= ncols) continue;
      int box, r;
      col_box(c0 + c, s.R, box, r);
      const cd gb = gbar[(((long long)pl * s.R + r) * nleaf + box) * ni + i];
      const cd x = make_double2(Out[e].x + gb.x, Out[e].y + gb.y);
      for (int kk = 0; kk < s.K; ++kk) acc[(c * s.K + kk) * ni + i] += cf[kk].x * x.x - cf[kk].y * x.y;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NC * s.K * ni; e += blockDim.x) {
    const int c = e / (s.K * ni), rem = e - c * s.K * ni, kk = rem / ni, i = rem - kk * ni;
    if (c0 + c >= ncols) continue;
    int box, r;
    col_box(c0 + c, s.R, box, r);
    part[(((long long)chunk * s.R + r) * s.K + kk) * s.n_int + (long long)box * ni + i] = acc[e];
  }
}

// wave: u_bar = A^T P1_bar - C0 y_u (A = c^2-weighted nested differentiation at
// interior rows, its transpose scattered onto the leaf's nodes), v_bar = P0_bar at
// interior nodes and 0 elsewhere.  out must hold u_bar = -C0 y_u, v_bar = 0 on entry.
__global__ void k_adj_post_wave(LeafGeo g, int R, long long n_nodes, int K, int nchunk,
                                const double* __restrict__ acoef, const double* __restrict__ part,
                                double* __restrict__ out) {
  const int leaf = blockIdx.x, r = blockIdx.y;
  const int a = leaf % g.nlx, b = leaf / g.nlx, p = g.p, q = g.q;
  extern __shared__ double sd[];
  double* P1 = sd;               // p x p, interior entries only
  double* al = sd + p * p;
  double* tx = sd + 2 * p * p;   // sum_k Dx[k,l] P1(k,j) at (l, j)
  double* ty = sd + 3 * p * p;   // sum_j Dy[j,l] P1(k,j) at (k, l)
  const long long ni = (long long)q * q;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int k = t % p, j = t / p;
    const long long id = gnode(g, a, b, k, j);
    al[t] = id < 0 ? 0.0 : acoef[id];
    double v0 = 0, v1 = 0;
    if (k > 0 && k < p - 1 && j > 0 && j < p - 1) {
      const long long o = (long long)leaf * ni + (j - 1) * q + (k - 1);
      for (int c = 0; c < nchunk; ++c) {
        v0 += part[(((long long)c * R + r) * K + 0) * g.n_int + o];
        v1 += part[(((long long)c * R + r) * K + 1) * g.n_int + o];
      }
      out[((long long)r * 2 + 1) * n_nodes + id] = v0;
    }
    P1[t] = v1;
  }
  __syncthreads();
  // forward: (A u)(k,j) = sum_l Dx[k,l] a(l,j) sum_m Dx[l,m] u(m,j) + same in y.
  // transpose: u_bar(m,j) += sum_l Dx[l,m] a(l,j) sum_k Dx[k,l] P1(k,j)  (and y)
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int l = t % p, j = t / p;
    double sx = 0, sy = 0;
    for (int k = 1; k < p - 1; ++k) sx += g.Dx[k * p + l] * P1[j * p + k];          // row j, column l
    const int kk = l, ll = j;                                                       // (k, l) = (t % p, t / p)
    for (int jj = 1; jj < p - 1; ++jj) sy += g.Dy[jj * p + ll] * P1[jj * p + kk];
    tx[t] = al[t] * sx;    // at (l, j)
    ty[t] = al[t] * sy;    // at (k, l) with k = t % p, l = t / p
  }
  __syncthreads();
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int m = t % p, j = t / p;
    const long long id = gnode(g, a, b, m, j);
    if (id < 0) continue;
    double v = 0;
    if (j > 0 && j < p - 1)
      for (int l = 0; l < p; ++l) v += g.Dx[l * p + m] * tx[j * p + l];
    if (m > 0 && m < p - 1)
      for (int l = 0; l < p; ++l) v += g.Dy[l * p + j] * ty[l * p + m];
    if (v != 0.0) atomicAdd(&out[(long long)r * 2 * n_nodes + id], v);
  }
}

__global__ void k_adj_init_wave(long long n_nodes, int R, double C0, const double* __restrict__ y,
                                double* __restrict__ out) {
  const long long tot = (long long)R * n_nodes;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / n_nodes, node = t - r * n_nodes;
    out[r * 2 * n_nodes + node] = -C0 * y[r * 2 * n_nodes + node];
    out[(r * 2 + 1) * n_nodes + node] = 0.0;
  }
}

// ---------------------------------------------------------------- shallow water
// Transpose of k_post_sw.  Forward, at every node the leaf owns:
//   U = C1 F1 + C2 F2 + tg (dx A1 + dy A2),  V = -C2 F1 + C1 F2 + tg (-dx A2 + dy A1),  h = A0,
// dx, dy the node-gradient stencils (leaf rows / columns inside, mean of the
// one-sided normal derivatives on interfaces, edge interpolant tangentially).
// Here every stencil weight is scattered back onto the accumulated fields
// abar[r][k][node] and the direct terms onto out (F1, F2 fields).
__device__ __forceinline__ void scat_dx(const LeafGeo& g, double* f, int a, int b, int k, int j, double w) {
  for (int m = 0; m < g.p; ++m) {
    const long long id = gnode(g, a, b, m, j);
    if (id >= 0) atomicAdd(&f[id], g.Dx[k * g.p + m] * w);
  }
}
__device__ __forceinline__ void scat_dy(const LeafGeo& g, double* f, int a, int b, int k, int j, double w) {
  for (int m = 0; m < g.p; ++m) {
    const long long id = gnode(g, a, b, k, m);
    if (id >= 0) atomicAdd(&f[id], g.Dy[j * g.p + m] * w);
  }
}

__global__ void k_adj_post_sw(LeafGeo g, int R, long long n_nodes, const double* __restrict__ y,
                              double* __restrict__ abar, double* __restrict__ out, double C1, double C2,
                              double taug) {
  const int leaf = blockIdx.x, r = blockIdx.y;
  const int a = leaf % g.nlx, b = leaf / g.nlx, p = g.p, q = g.q;
  const double* yr = y + (long long)r * 3 * n_nodes;
  double* ab0 = abar + (long long)r * 3 * n_nodes;
  double* ab1 = ab0 + n_nodes;
  double* ab2 = ab1 + n_nodes;
  double* o = out + (long long)r * 3 * n_nodes;
  auto direct = [&](long long id, double& s1x, double& s1y, double& s2x, double& s2y) {
    const double yU = yr[id], yV = yr[n_nodes + id], yh = yr[2 * n_nodes + id];
    atomicAdd(&ab0[id], yh);
    atomicAdd(&o[id], C1 * yU - C2 * yV);
    atomicAdd(&o[n_nodes + id], C2 * yU + C1 * yV);
    s1x = taug * yU;  // weight of dx A1
    s1y = taug * yV;  // dy A1
    s2x = -taug * yV; // dx A2
    s2y = taug * yU;  // dy A2
  };
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) {
    const int k = t % q + 1, j = t / q + 1;
    double s1x, s1y, s2x, s2y;
    direct(gnode(g, a, b, k, j), s1x, s1y, s2x, s2y);
    scat_dx(g, ab1, a, b, k, j, s1x);
    scat_dy(g, ab1, a, b, k, j, s1y);
    scat_dx(g, ab2, a, b, k, j, s2x);
    scat_dy(g, ab2, a, b, k, j, s2y);
  }
  for (int t = threadIdx.x; t < 4 * q; t += blockDim.x) {
    const int side = t / q, oo = t % q + 1;
    if (side == 1 && a != g.nlx - 1) continue;
    if (side == 2 && b != g.nly - 1) continue;
    double s1x, s1y, s2x, s2y;
    if (side == 0 || side == 2) {                // normal y, tangential x
      const int j = side == 0 ? 0 : p - 1, k = oo;
      direct(gnode(g, a, b, k, j), s1x, s1y, s2x, s2y);
      const double wn = (side == 0 && b > 0) ? 0.5 : 1.0;
      scat_dy(g, ab1, a, b, k, j, wn * s1y);
      scat_dy(g, ab2, a, b, k, j, wn * s2y);
      if (side == 0 && b > 0) {
        scat_dy(g, ab1, a, b - 1, k, p - 1, 0.5 * s1y);
        scat_dy(g, ab2, a, b - 1, k, p - 1, 0.5 * s2y);
      }
      for (int m = 1; m <= q; ++m) {
        const long long id = gnode(g, a, b, m, j);
        atomicAdd(&ab1[id], g.Ex[(k - 1) * q + (m - 1)] * s1x);
        atomicAdd(&ab2[id], g.Ex[(k - 1) * q + (m - 1)] * s2x);
      }
    } else {                                     // normal x, tangential y
      const int k = side == 3 ? 0 : p - 1, j = oo;
      direct(gnode(g, a, b, k, j), s1x, s1y, s2x, s2y);
      const double wn = (side == 3 && a > 0) ? 0.5 : 1.0;
      scat_dx(g, ab1, a, b, k, j, wn * s1x);
      scat_dx(g, ab2, a, b, k, j, wn * s2x);
      if (side == 3 && a > 0) {
        scat_dx(g, ab1, a - 1, b, p - 1, j, 0.5 * s1x);
        scat_dx(g, ab2, a - 1, b, p - 1, j, 0.5 * s2x);
      }
      for (int m = 1; m <= q; ++m) {
        const long long id = gnode(g, a, b, k, m);
        atomicAdd(&ab1[id], g.Ey[(j - 1) * q + (m - 1)] * s1y);
        atomicAdd(&ab2[id], g.Ey[(j - 1) * q + (m - 1)] * s2y);
      }
    }
  }
}

// Root wall solve transposed: qbar = Binv^T e_bar(wall); h_bar_root = -nu qbar;
// qbar kept per pole for the wall right-hand side's dependence on (F1, F2).
template <int NC, typename TA>
__global__ void __launch_bounds__(256) k_adj_root_sw(Sweep s, RootArgs ra, const cd* __restrict__ E,
                                                     cd* __restrict__ hroot, cd* __restrict__ qbar) {
  extern __shared__ cd smem[];
  const int pl = blockIdx.y, p = s.p0 + pl;
  const int c0 = blockIdx.x * NC;
  const int n = ra.n;
  TA* Xs = (TA*)smem;
  cd* Out = after(Xs, (size_t)NC * n);
  const int nq = ra.nq;
  for (int e = threadIdx.x; e < NC * n; e += blockDim.x) {
    const int c = e / n, i = e - c * n;
    cd v = make_double2(0.0, 0.0);
    if (c0 + c < s.R) v = E[((long long)pl * s.R + c0 + c) * s.n_edge + (long long)ra.bseg[i / ra.q] * ra.q + (i % ra.q)];
    if (nq) Out[e] = v;
    else Xs[e] = Cv<TA>::from(v);
  }
  __syncthreads();
  if (nq) {
    // (B^{-1})^T = D P^T H^T diag(Chat_m^{-T}) G^T P (the forward kernel's factors
    // transposed): zhat_m[s] = sum_k i^{mk} x[idx_k(s)], then the transposed blocks
    for (int e = threadIdx.x; e < NC * n; e += blockDim.x) {
      const int c = e / n, rem = e - c * n, m = rem / nq, sr = rem - m * nq;
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const cd v = times_ipow(Out[c * n + ra.c4idx[k * nq + sr]], m * k);
        re += v.x;
        im += v.y;
      }
      Xs[e] = Cv<TA>::from(make_double2(re, im));
    }
    __syncthreads();
    const TA* A = (const TA*)ra.Binv + (long long)p * 4 * nq * nq;
    for (int m = 0; m < 4; ++m)
      cmvT<NC, TA>(A + (long long)m * nq * nq, nq, nq, nq, Xs + m * nq, n, Out + (size_t)m * NC * nq);
  } else {
    cmvT<NC, TA>((const TA*)ra.Binv + (long long)p * n * n, n, n, n, Xs, n, Out);
  }
  for (int e = threadIdx.x; e < NC * n; e += blockDim.x) {
    const int c = e / n, j = e - c * n;
    const int r = c0 + c;
    if (r >= s.R) continue;
    int side;
    if (j < ra.sxq) side = 0;
    else if (j < ra.sxq + ra.syq) side = 1;
    else if (j < 2 * ra.sxq + ra.syq) side = 2;
    else side = 3;
    cd qv;
    if (nq) {
      // out[idx_k(s)] = c4_sign(k) (1/4) sum_m (-i)^{mk} zhat'_m[s]
      const int ks = ra.c4inv[j], k = ks / nq, sr = ks - k * nq;
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const cd v = times_ipow(Out[((size_t)m * NC + c) * nq + sr], -(m * k));
        re += v.x;
        im += v.y;
      }
      qv = make_double2(0.25 * c4_sign(k) * re, 0.25 * c4_sign(k) * im);
    } else {
      qv = Out[e];
    }
    const cd nu = ra.nu[p * 4 + side];
    const cd hv = cmul(nu, qv);
    const long long o = ((long long)pl * s.R + r) * n + j;
    qbar[o] = qv;
    hroot[o] = make_double2(-hv.x, -hv.y);
  }
}

// wall right-hand side transposed, summed over poles in order:
// F1 += Re sum_p b0_p qbar_p, F2 += Re sum_p b1_p qbar_p at wall nodes
__global__ void k_adj_root_rhs(Sweep s, RootArgs ra, const cd* __restrict__ qbar, double* __restrict__ out) {
  const int n = ra.n;
  const long long tot = (long long)s.R * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / n), j = (int)(t % n);
    int side;
    if (j < ra.sxq) side = 0;
    else if (j < ra.sxq + ra.syq) side = 1;
    else if (j < 2 * ra.sxq + ra.syq) side = 2;
    else side = 3;
    double f1 = 0, f2 = 0;
    for (int pl = 0; pl < s.P; ++pl) {
      const int p = s.p0 + pl;
      const cd qv = qbar[((long long)pl * s.R + r) * n + j];
      const cd b0 = ra.bcoef[(p * 4 + side) * 2], b1 = ra.bcoef[(p * 4 + side) * 2 + 1];
      f1 += b0.x * qv.x - b0.y * qv.y;
      f2 += b1.x * qv.x - b1.y * qv.y;
    }
    const long long node = s.n_int + (long long)ra.bseg[j / ra.q] * ra.q + (j % ra.q);
    atomicAdd(&out[(long long)r * 3 * s.n_nodes + node], f1);
    atomicAdd(&out[((long long)r * 3 + 1) * s.n_nodes + node], f2);
  }
}

// Pre-map transposed: r_bar = P0 at interior; div F and curl F are leaf
// derivatives at interior nodes, so F1 += dx^T P1 - dy^T P2, F2 += dy^T P1 + dx^T P2.
__global__ void k_adj_pre_sw(LeafGeo g, int R, long long n_nodes, int K, int nchunk,
                             const double* __restrict__ part, double* __restrict__ out) {
  const int leaf = blockIdx.x, r = blockIdx.y;
  const int a = leaf % g.nlx, b = leaf / g.nlx, q = g.q;
  const long long ni = (long long)q * q;
  double* o1 = out + (long long)r * 3 * n_nodes;
  double* o2 = o1 + n_nodes;
  double* oh = o2 + n_nodes;
  for (int t = threadIdx.x; t < q * q; t += blockDim.x) {
    const int k = t % q + 1, j = t / q + 1;
    const long long o = (long long)leaf * ni + t;
    double P0 = 0, P1 = 0, P2 = 0;
    for (int c = 0; c < nchunk; ++c) {
      P0 += part[(((long long)c * R + r) * K + 0) * g.n_int + o];
      P1 += part[(((long long)c * R + r) * K + 1) * g.n_int + o];
      P2 += part[(((long long)c * R + r) * K + 2) * g.n_int + o];
    }
    atomicAdd(&oh[gnode(g, a, b, k, j)], P0);
    scat_dx(g, o1, a, b, k, j, P1);
    scat_dy(g, o1, a, b, k, j, -P2);
    scat_dy(g, o2, a, b, k, j, P1);
    scat_dx(g, o2, a, b, k, j, P2);
  }
}

// ---------------------------------------------------------------- host driver
namespace {

int pick_nc_t(int shared, int R, int k, int rows, int nbox = 1 << 30) {
  int nc = 1;
  if (shared) {
    const long long ncols = (long long)nbox * R;
    while (nc < 8 && 2 * nc <= ncols) nc *= 2;
  } else {
    while (nc < 8 && R % (nc * 2) == 0) nc *= 2;
  }
  while (nc > 1 && (size_t)nc * (k + rows + 64) * sizeof(cd) > 200 * 1024) nc /= 2;
  return nc;
}

#define EO_SET_SMEM_T(kern, bytes)                                                            \
  do {                                                                                        \
    /* raise the dynamic shared-memory cap once per kernel and device */                     \
    static size_t cap_[64] = {};                                                              \
    eo_status rs_ = ensure_smem((const void*)(kern), (bytes), cap_, 200 * 1024 + 8192);       \
    if (rs_) return rs_;                                                                      \
  } while (0)

template <int NC, typename TA>
struct AdjDownLeaf {
  static eo_status run(const Sweep& s, const Handle& h, int nleaf, cd* gbar, cd* ybar, cudaStream_t st) {
    dim3 grid((nleaf * s.R + NC - 1) / NC, s.P);
    const size_t smem = sizeof(cd) * ((size_t)NC * (2 * s.ni + s.nb)) + 64;
    EO_SET_SMEM_T((k_adj_down_leaf<NC, TA>), smem);
    k_adj_down_leaf<NC, TA><<<grid, 256, smem, st>>>(s, h.aXY, h.xy_pstride, h.xy_bstride, nleaf, gbar, ybar);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct AdjDownMerge {
  static eo_status run(const Sweep& s, const MergeArgs& m, cd* E, cudaStream_t st) {
    dim3 grid((m.nbox * s.R + NC - 1) / NC, s.P);
    const size_t smem = sizeof(cd) * ((size_t)NC * (m.n3 + m.nbd)) + 64;
    EO_SET_SMEM_T((k_adj_down_merge<NC, TA>), smem);
    k_adj_down_merge<NC, TA><<<grid, 256, smem, st>>>(s, m, E);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct AdjUpMerge {
  static eo_status run(const Sweep& s, const MergeArgs& m, const cd* hpar, cd* hchild, cudaStream_t st) {
    dim3 grid((m.nbox * s.R + NC - 1) / NC, s.P);
    const size_t smem = sizeof(cd) * ((size_t)NC * (m.zu_rows + m.n3)) + 64;
    EO_SET_SMEM_T((k_adj_up_merge<NC, TA>), smem);
    k_adj_up_merge<NC, TA><<<grid, 256, smem, st>>>(s, m, hpar, hchild);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct AdjUpLeaf {
  static eo_status run(const Sweep& s, const Handle& h, int nleaf, int nchunk, int ppc, const cd* h0,
                       const cd* gbar, double* part, cudaStream_t st) {
    dim3 grid((nleaf * s.R + NC - 1) / NC, nchunk);
    const size_t smem = sizeof(cd) * ((size_t)NC * (s.nb + s.ni)) + sizeof(double) * NC * s.K * s.ni + 64;
    EO_SET_SMEM_T((k_adj_up_leaf<NC, TA>), smem);
    k_adj_up_leaf<NC, TA><<<grid, 256, smem, st>>>(s, h.aH, h.h_pstride, h.h_bstride, nleaf, ppc, h0, gbar, part);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <int NC, typename TA>
struct AdjRootSW {
  static eo_status run(const Sweep& s, const RootArgs& ra, const cd* E, cd* hroot, cd* qbar, cudaStream_t st) {
    dim3 grid((s.R + NC - 1) / NC, s.P);
    const size_t smem = sizeof(cd) * ((size_t)NC * 2 * ra.n) + 64;
    EO_SET_SMEM_T((k_adj_root_sw<NC, TA>), smem);
    k_adj_root_sw<NC, TA><<<grid, 256, smem, st>>>(s, ra, E, hroot, qbar);
    EO_CUDA_TRY(cudaGetLastError());
    return EO_OK;
  }
};

template <template <int, typename> class Launcher, typename TA, typename... Args>
eo_status dispatch_nc_t(int nc, Args&&... args) {
  switch (nc) {
    case 1: return Launcher<1, TA>::run(args...);
    case 2: return Launcher<2, TA>::run(args...);
    case 4: return Launcher<4, TA>::run(args...);
    default: return Launcher<8, TA>::run(args...);
  }
}

template <template <int, typename> class Launcher, typename... Args>
eo_status dispatch_t(int prec, int nc, Args&&... args) {
  if (prec == 1) return dispatch_nc_t<Launcher, float2>(nc, args...);
  if (prec == 2) return dispatch_nc_t<Launcher, float4>(nc, args...);
  return dispatch_nc_t<Launcher, double2>(nc, args...);
}

MergeArgs merge_args_t(const Handle& h, int l) {
  const LevelDev& ld = h.lv[l];
  const LevelDev& lc = h.lv[l - 1];
  MergeArgs m;
  m.nbox = ld.nbox; m.nbx = ld.nbx; m.nbx_c = lc.nbx; m.nbox_c = lc.nbox; m.dir = ld.dir;
  m.nbd = ld.nbd; m.nbd_c = lc.nbd; m.n3 = ld.n3; m.zu_rows = ld.zu_rows;
  m.par_child = ld.par_child; m.par_idx = ld.par_idx; m.a3 = ld.a3; m.b3 = ld.b3;
  m.ZU = ld.aZU; m.zps = ld.zu_pstride; m.zbs = ld.zu_bstride;
  m.S = ld.aS; m.sps = ld.s_pstride; m.sbs = ld.s_bstride;
  m.bseg = ld.bseg; m.iseg = ld.iseg; m.nseg = ld.nseg; m.w3 = ld.w3;
  return m;
}

eo_status adjoint_step(Handle& h, const double* yin, double* yout, int R, cudaStream_t st) {
  const Grid& g = h.g;
  const int q = g.q, ni = q * q, nb = 4 * q;
  const int nleaf = g.nlx * g.nly;
  const int L = h.plan.L();
  eo_status rc;
  Sweep s;
  s.R = R; s.P = h.P; s.p0 = 0; s.q = q; s.ni = ni; s.nb = nb;
  s.n_int = g.n_int; s.n_edge = g.n_edge; s.n_nodes = g.n_nodes; s.shared = h.shared;
  s.K = h.K; s.coef = h.coef; s.wgt = h.wgt;
  LeafGeo geo{g.nlx, g.nly, g.p, q, g.n_int, g.n_hseg, h.dDx, h.dDx + g.p * g.p, h.dDx + 2 * g.p * g.p,
              h.dDx + 2 * g.p * g.p + q * q};
  const bool sw = h.kind == EO_SW_WALLS;
  if (!sw) {
    // seeds: forward accumulators A0 -> v, A1 -> u
    s.src[0] = yin + g.n_nodes; s.src_rs[0] = 2 * g.n_nodes;
    s.src[1] = yin;             s.src_rs[1] = 2 * g.n_nodes;
  } else {
    // post-map transposed onto the accumulated fields (abar) and the direct terms
    EO_CUDA_TRY(cudaMemsetAsync(yout, 0, sizeof(double) * (size_t)R * 3 * g.n_nodes, st));
    EO_CUDA_TRY(cudaMemsetAsync(h.abar, 0, sizeof(double) * (size_t)R * 3 * g.n_nodes, st));
    if ((rc = h.trace_begin(st))) return rc;
    k_adj_post_sw<<<dim3(nleaf, R), 128, 0, st>>>(geo, R, g.n_nodes, yin, h.abar, yout, h.C[0], h.C[1],
                                                   h.tau * h.opts.sw_g);
    EO_CUDA_TRY(cudaGetLastError());
    if ((rc = h.trace_end(TR_POST, st))) return rc;
    for (int k = 0; k < 3; ++k) { s.src[k] = h.abar + k * g.n_nodes; s.src_rs[k] = 3 * g.n_nodes; }
  }
  cd* ybar = h.hB;
  if ((rc = h.trace_begin(st))) return rc;
  if ((rc = dispatch_t<AdjDownLeaf>(h.fp32, pick_nc_t(h.shared, R, ni + nb, ni, nleaf), s, h, nleaf, h.gbar, ybar, st)))
    return rc;
  if ((rc = h.trace_end(TR_DOWN_LEAF, st))) return rc;
  if ((rc = h.trace_begin(st))) return rc;
  k_adj_edges<<<(unsigned)std::min<long long>(8192, ((long long)h.P * R * g.n_edge + 255) / 256), 256, 0, st>>>(
      s, g.nlx, g.nly, ybar, h.E);
  EO_CUDA_TRY(cudaGetLastError());
  if ((rc = h.trace_end(TR_EDGE, st))) return rc;
  for (int l = 1; l <= L; ++l) {
    MergeArgs m = merge_args_t(h, l);
    if ((rc = h.trace_begin(st))) return rc;
    if ((rc = dispatch_t<AdjDownMerge>(h.lv[l].fp32, pick_nc_t(h.shared, R, m.nbd, m.n3, m.nbox), s, m, h.E, st))) return rc;
    if ((rc = h.trace_end(TR_DOWN_MERGE, st))) return rc;
  }
  cd* hpar = h.hA;
  cd* hch = h.hB;
  if (sw) {
    // wall solve transposed: h_bar at the root and the wall rhs's dependence on F
    const Level& rl = h.plan.lv[L];
    RootArgs ra{rl.nbd, q, rl.sx * q, rl.sy * q, h.lv[L].bseg, h.aBinv, h.bcoef, h.nu, yin, 3,
                h.c4, h.c4idx, h.c4inv};
    if ((rc = h.trace_begin(st))) return rc;
    if ((rc = dispatch_t<AdjRootSW>(h.root_fp32, pick_nc_t(0, R, rl.nbd, rl.nbd), s, ra, h.E, hpar, h.qbar, st)))
      return rc;
    k_adj_root_rhs<<<(unsigned)std::min<long long>(4096, ((long long)R * rl.nbd + 255) / 256), 256, 0, st>>>(
        s, ra, h.qbar, yout);
    EO_CUDA_TRY(cudaGetLastError());
    if ((rc = h.trace_end(TR_ROOT, st))) return rc;
  } else if (L == 0) {  // one leaf: its boundary is the wall, no flux seeds reach it
    EO_CUDA_TRY(cudaMemsetAsync(hpar, 0, sizeof(cd) * (size_t)h.P * R * nleaf * nb, st));
  }
  for (int l = L; l >= 1; --l) {
    MergeArgs m = merge_args_t(h, l);
    if ((rc = h.trace_begin(st))) return rc;
    if ((rc = dispatch_t<AdjUpMerge>(h.lv[l].fp32, pick_nc_t(h.shared, R, m.n3, m.zu_rows, m.nbox), s, m, hpar, hch, st)))
      return rc;
    if ((rc = h.trace_end(TR_UP_MERGE, st))) return rc;
    std::swap(hpar, hch);
  }
  const int nc = pick_nc_t(h.shared, R, ni, nb, nleaf);
  const int ncg = (nleaf * R + nc - 1) / nc;
  int nchunk = std::max(1, std::min(h.P, (608 + ncg - 1) / ncg));
  nchunk = std::min(nchunk, h.nchunk);
  const int ppc = (h.P + nchunk - 1) / nchunk;
  nchunk = (h.P + ppc - 1) / ppc;
  if ((rc = h.trace_begin(st))) return rc;
  if ((rc = dispatch_t<AdjUpLeaf>(h.fp32, nc, s, h, nleaf, nchunk, ppc, hpar, h.gbar, h.part, st))) return rc;
  if ((rc = h.trace_end(TR_UP_LEAF, st))) return rc;
  if (sw) {
    if ((rc = h.trace_begin(st))) return rc;
    k_adj_pre_sw<<<dim3(nleaf, R), 128, 0, st>>>(geo, R, g.n_nodes, h.K, nchunk, h.part, yout);
    EO_CUDA_TRY(cudaGetLastError());
    if ((rc = h.trace_end(TR_PRE, st))) return rc;
    return EO_OK;
  }
  if ((rc = h.trace_begin(st))) return rc;
  k_adj_init_wave<<<(unsigned)std::min<long long>(8192, ((long long)R * g.n_nodes + 255) / 256), 256, 0, st>>>(
      g.n_nodes, R, h.C[0], yin, yout);
  EO_CUDA_TRY(cudaGetLastError());
  k_adj_post_wave<<<dim3(nleaf, R), 128, sizeof(double) * 4 * g.p * g.p, st>>>(geo, R, g.n_nodes, h.K, nchunk,
                                                                              h.acoef, h.part, yout);
  EO_CUDA_TRY(cudaGetLastError());
  if ((rc = h.trace_end(TR_POST, st))) return rc;
  return EO_OK;
}

}  // namespace

eo_status apply_adjoint(Handle& h, double* y, int n_rhs, int n_steps, cudaStream_t st) {
  if (!y) return fail(EO_ERR_INVALID_ARG, "null state");
  if (n_rhs < 1 || n_rhs > h.R) return fail(EO_ERR_INVALID_ARG, "n_rhs out of range [1, max_rhs]");
  if (n_steps < 0) return fail(EO_ERR_INVALID_ARG, "negative n_steps");
  if (!h.gbar) {
    eo_status rc = h.alloc((void**)&h.gbar, sizeof(cd) * (size_t)h.P * h.R * h.g.n_int, false);
    if (rc) return rc;
    if (h.kind == EO_SW_WALLS) {
      if ((rc = h.alloc((void**)&h.abar, sizeof(double) * (size_t)h.R * 3 * h.g.n_nodes, false))) return rc;
      if ((rc = h.alloc((void**)&h.qbar, sizeof(cd) * (size_t)h.P * h.R * h.nroot, false))) return rc;
    }
  }
  double* cur = y;
  double* nxt = h.ustate;
  eo_status rc;
  for (int i = 0; i < n_steps; ++i) {
    if ((rc = adjoint_step(h, cur, nxt, n_rhs, st))) return rc;
    std::swap(cur, nxt);
  }
  if (cur != y)
    EO_CUDA_TRY(cudaMemcpyAsync(y, cur, sizeof(double) * (size_t)n_rhs * h.F * h.g.n_nodes,
                                cudaMemcpyDeviceToDevice, st));
  return EO_OK;
}

}  // namespace eo
