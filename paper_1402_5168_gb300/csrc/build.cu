// Build phase (Section 1.3 and Section 2.3), FP64 on the device.
//
// For every distinct pole alpha (Im alpha >= 0; the conjugates follow from
// eq. "conjugate, matrix inverses" of Section 3.3) the elliptic problem
//     div(a grad w) - kappa^2 w = s        (Section 2.1)
// is discretised by Chebyshev collocation on every leaf (Section 2.2) and
// solved by nested dissection:
//   leaf:  A_ii [X | Y] = [I | -A_ib]  (interior rows, boundary data u_b)
//          T = F_bb + F_bi Y  (outward flux a dw/dn from boundary data)
//          H = F_bi X         (outward flux of the particular solution)
//   merge of boxes alpha, beta over interface 3 (flux continuity):
//          Z = (T^a_33 + T^b_33)^{-1},  S = -Z [T^a_31 | T^b_32],
//          U = -[T^a_13 ; T^b_23] Z,    T_parent = diag(T^a_11, T^b_22) + [T^a_13; T^b_23] S
//   root:  Dirichlet walls: boundary data 0, only Z is kept.
//          Shallow-water walls: the oblique condition of the walls, written
//          with T_root, is inverted once per pole (B_root^{-1}).
// Dense factorisations and products of the build call cuBLAS batched routines;
// assembly and gathers are the kernels below.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "handle.h"

namespace eo {

#define EO_CUBLAS_TRY(expr)                                                     \
  do {                                                                          \
    cublasStatus_t s_ = (expr);                                                 \
    if (s_ != CUBLAS_STATUS_SUCCESS)                                            \
      return fail(EO_ERR_CUDA, std::string(#expr) + ": cublas status " + std::to_string((int)s_)); \
  } while (0)

// local boundary index of leaf node (k, j) in S, E, N, W order; -1 if interior
__device__ __forceinline__ int bidx(int k, int j, int p, int q) {
  if (j == 0) return k - 1;
  if (k == p - 1) return q + j - 1;
  if (j == p - 1) return 2 * q + k - 1;
  if (k == 0) return 3 * q + j - 1;
  return -1;
}

// global node id of local node (k, j) of leaf (a, b); per: periodic square, whose
// top / right edge lines are lines 0
__device__ __forceinline__ long long dnode(int a, int b, int k, int j, int nlx, int nly, int p,
                                           long long n_int, long long n_hseg, int per) {
  const int q = p - 2;
  const bool kin = k > 0 && k < p - 1, jin = j > 0 && j < p - 1;
  if (kin && jin) return ((long long)b * nlx + a) * q * q + (long long)(j - 1) * q + (k - 1);
  if (kin) return n_int + ((long long)(j == 0 ? b : ((per && b + 1 == nly) ? 0 : b + 1)) * nlx + a) * q + (k - 1);
  if (jin) {
    const int nvl = per ? nlx : nlx + 1;
    return n_int + (n_hseg + (long long)b * nvl + (k == 0 ? a : ((per && a + 1 == nlx) ? 0 : a + 1))) * q + (j - 1);
  }
  return -1;
}

// Real leaf matrices, column-major: Aii0 (n_i x n_i), Aib (n_i x n_b),
// Fbi (n_b x n_i), Fbb (n_b x n_b).  One block per leaf.
__global__ void leaf_real_ops(int nlx, int nly, int p, long long n_int, long long n_hseg, int per,
                              const double* __restrict__ Dx, const double* __restrict__ Dy,
                              const double* __restrict__ acoef, double* Aii0, double* Aib,
                              double* Fbi, double* Fbb) {
  const int leaf = blockIdx.x;
  const int a = leaf % nlx, b = leaf / nlx;
  const int q = p - 2, ni = q * q, nb = 4 * q;
  extern __shared__ double sm[];
  double* al = sm;   // a at local nodes, [j*p + k]
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int k = t % p, j = t / p;
    const long long id = dnode(a, b, k, j, nlx, nly, p, n_int, n_hseg, per);
    al[t] = (id < 0) ? 0.0 : (acoef ? acoef[id] : 1.0);
  }
  __syncthreads();
  double* A0 = Aii0 + (size_t)leaf * ni * ni;
  double* Ab = Aib + (size_t)leaf * ni * nb;
  double* Fi = Fbi + (size_t)leaf * nb * ni;
  double* Fb = Fbb + (size_t)leaf * nb * nb;
  // interior rows: d/dx(a du/dx) + d/dy(a du/dy) with nested 1-D differentiation
  for (int r = threadIdx.x; r < ni; r += blockDim.x) {
    const int k = r % q + 1, j = r / q + 1;
    for (int m = 0; m < p; ++m) {
      double cx = 0, cy = 0;
      for (int l = 0; l < p; ++l) {
        cx += Dx[k * p + l] * al[j * p + l] * Dx[l * p + m];
        cy += Dy[j * p + l] * al[l * p + k] * Dy[l * p + m];
      }
      // x part: column (m, j); y part: column (k, m)
      int bi = bidx(m, j, p, q);
      if (bi < 0) A0[r + (size_t)((j - 1) * q + (m - 1)) * ni] += cx;
      else Ab[r + (size_t)bi * ni] += cx;
      bi = bidx(k, m, p, q);
      if (bi < 0) A0[r + (size_t)((m - 1) * q + (k - 1)) * ni] += cy;
      else Ab[r + (size_t)bi * ni] += cy;
    }
  }
  // boundary rows: outward flux a dw/dn by one-sided spectral differentiation
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    const int side = t / q, o = t % q + 1;
    for (int m = 0; m < p; ++m) {
      int k, j;
      double c;
      if (side == 0) { k = o; j = m; c = -al[0 * p + o] * Dy[0 * p + m]; }
      else if (side == 1) { k = m; j = o; c = al[o * p + (p - 1)] * Dx[(p - 1) * p + m]; }
      else if (side == 2) { k = o; j = m; c = al[(p - 1) * p + o] * Dy[(p - 1) * p + m]; }
      else { k = m; j = o; c = -al[o * p + 0] * Dx[0 * p + m]; }
      const int bi = bidx(k, j, p, q);
      if (bi < 0) Fi[t + (size_t)((j - 1) * q + (k - 1)) * nb] += c;
      else Fb[t + (size_t)bi * nb] += c;
    }
  }
}

// Leaf coupling of Curl(G h) to the leaf's own edge values (shallow water,
// consistent elimination), column-major ni x nb like Aib.  At interior node (k, j):
//   Curl(G h) = Dy[j][0] (dX h_S)(k) + Dy[j][p-1] (dX h_N)(k)
//             - Dx[k][0] (dY h_W)(j) - Dx[k][p-1] (dY h_E)(j),
// dX = (Dx)_{interior} - Ex and dY = (Dy)_{interior} - Ey: the difference between the
// leaf's own differentiation along an edge (corner columns dropped) and the edge
// interpolant's derivative used by the recovered gradient.  One block per leaf.
__global__ void leaf_curl_ops(int p, const double* __restrict__ Dx, const double* __restrict__ Dy,
                              const double* __restrict__ Ex, const double* __restrict__ Ey, double* Cib) {
  const int q = p - 2, ni = q * q;
  double* C = Cib + (size_t)blockIdx.x * ni * 4 * q;
  for (int r = threadIdx.x; r < ni; r += blockDim.x) {
    const int k = r % q + 1, j = r / q + 1;
    for (int m = 1; m <= q; ++m) {
      const double dX = Dx[k * p + m] - Ex[(k - 1) * q + (m - 1)];
      const double dY = Dy[j * p + m] - Ey[(j - 1) * q + (m - 1)];
      C[r + (size_t)(m - 1) * ni] = Dy[j * p + 0] * dX;                   // S node (m, 0)
      C[r + (size_t)(2 * q + m - 1) * ni] = Dy[j * p + (p - 1)] * dX;     // N node (m, p-1)
      C[r + (size_t)(3 * q + m - 1) * ni] = -Dx[k * p + 0] * dY;          // W node (0, m)
      C[r + (size_t)(q + m - 1) * ni] = -Dx[k * p + (p - 1)] * dY;        // E node (p-1, m)
    }
  }
}

// Batch entry i = (pole gi, leaf) with leaf = i % nleaf, gi = i / nleaf:
// A = Aii0 - kappa2[gi] I; XY = [I | -Aib]; T = Fbb (complex).
// With Cib (consistent shallow water): Y's right-hand side is -(Aib + beta[gi] Cib).
// With hw (per-box operators, a weight per interior node, leaf-major like the public
// interior numbering): the shift is kappa2[gi] diag(hw) instead.
__global__ void leaf_assemble(int nbatch, int nleaf, int ni, int nb, const cd* __restrict__ kappa2,
                              const double* Aii0, const double* Aib, const double* Fbb, const double* Cib,
                              const cd* __restrict__ beta, const double* __restrict__ hw, cd* A, cd* XY,
                              cd* T) {
  const size_t nA = (size_t)ni * ni, nXY = (size_t)ni * (ni + nb), nT = (size_t)nb * nb;
  const size_t tot = (size_t)nbatch * (nA + nXY + nT);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t bi = t / (nA + nXY + nT);
    size_t e = t % (nA + nXY + nT);
    const size_t leaf = bi % nleaf;
    if (e < nA) {
      const int i = e % ni, j = e / ni;
      const cd k2 = kappa2[bi / nleaf];
      const double wt = hw ? hw[leaf * ni + i] : 1.0;
      const double v = Aii0[leaf * nA + e];
      A[bi * nA + e] = make_double2(v - (i == j ? wt * k2.x : 0.0), (i == j ? -wt * k2.y : 0.0));
    } else if (e < nA + nXY) {
      e -= nA;
      const int i = e % ni, j = e / ni;
      if (j < ni) {
        XY[bi * nXY + e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      } else {
        const size_t o = leaf * (size_t)ni * nb + (e - (size_t)ni * ni);
        double re = -Aib[o], im = 0.0;
        if (Cib) {
          const cd bt = beta[bi / nleaf];
          re -= bt.x * Cib[o];
          im -= bt.y * Cib[o];
        }
        XY[bi * nXY + e] = make_double2(re, im);
      }
    } else {
      e -= nA + nXY;
      T[bi * nT + e] = make_double2(Fbb[leaf * nT + e], 0.0);
    }
  }
}

__global__ void real_to_complex(size_t n, const double* x, cd* y) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = make_double2(x[t], 0.0);
}

// Merge gathers for one level, one parent box per block (column-major outputs).
// Block index = gi * nbo + box: pole gi of the group, parent box (0 when shared).
// Children's T: Tc[gi][child box][nbd_c x nbd_c], nbo_c child blocks per pole.
__global__ void merge_gather(int nbd_c, int n3, int npar, const int* __restrict__ par_child,
                             const int* __restrict__ par_idx, const int* __restrict__ a3,
                             const int* __restrict__ b3, int dir, int nbx_par, int nbx_child,
                             int shared, int nbo, int nbo_c, const cd* __restrict__ Tc, cd* M33, cd* Q,
                             cd* Rm, cd* Tpar) {
  const int box = blockIdx.x % nbo, gi = blockIdx.x / nbo;
  int ca, cb;
  if (shared) { ca = cb = 0; }
  else {
    const int bx = box % nbx_par, by = box / nbx_par;
    if (dir == 0) { ca = by * nbx_child + 2 * bx; cb = ca + 1; }
    else { ca = (2 * by) * nbx_child + bx; cb = ca + nbx_child; }
  }
  const size_t nT = (size_t)nbd_c * nbd_c;
  const cd* Ta = Tc + ((size_t)gi * nbo_c + ca) * nT;
  const cd* Tb = Tc + ((size_t)gi * nbo_c + cb) * nT;
  const int box_out = blockIdx.x;
  cd* m33 = M33 + (size_t)box_out * n3 * n3;
  cd* qq = Q ? Q + (size_t)box_out * npar * n3 : nullptr;
  cd* rm = Rm + (size_t)box_out * n3 * npar;
  cd* tp = Tpar ? Tpar + (size_t)box_out * npar * npar : nullptr;
  for (int e = threadIdx.x; e < n3 * n3; e += blockDim.x) {
    const int t = e % n3, u = e / n3;
    cd x = Ta[a3[t] + (size_t)a3[u] * nbd_c], y = Tb[b3[t] + (size_t)b3[u] * nbd_c];
    m33[e] = make_double2(x.x + y.x, x.y + y.y);
  }
  if (!Q) return;
  for (int e = threadIdx.x; e < npar * n3; e += blockDim.x) {
    const int i = e % npar, t = e / npar;
    const int c = par_child[i], ci = par_idx[i];
    const cd* Tx = c ? Tb : Ta;
    const int c3 = c ? b3[t] : a3[t];
    qq[e] = Tx[ci + (size_t)c3 * nbd_c];                      // Q[i, t]
    rm[t + (size_t)i * n3] = Tx[c3 + (size_t)ci * nbd_c];     // Rm[t, i]
  }
  if (!tp) return;
  for (size_t e = threadIdx.x; e < (size_t)npar * npar; e += blockDim.x) {
    const int i = e % npar, ii = e / npar;
    const int c = par_child[i];
    tp[e] = (c == par_child[ii]) ? (c ? Tb : Ta)[par_idx[i] + (size_t)par_idx[ii] * nbd_c]
                                 : make_double2(0.0, 0.0);
  }
}

// dst (ldd) rows [0, n) x cols [0, n) = scale * src (n x n, ld n); batched over blocks
__global__ void copy_scaled(int n, const cd* src, cd* dst, int ldd, int64_t dst_stride, double scale) {
  const cd* s = src + (size_t)blockIdx.x * n * n;
  cd* d = dst + (size_t)blockIdx.x * dst_stride;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    d[i + (size_t)j * ldd] = make_double2(scale * s[e].x, scale * s[e].y);
  }
}

__global__ void set_identity(int n, int nbatch, cd* M) {
  const size_t tot = (size_t)nbatch * n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const size_t e = t % ((size_t)n * n);
    M[t] = make_double2((e % n) == (e / n) ? 1.0 : 0.0, 0.0);
  }
}

// B_root = diag(nu) T_root + tau f G_t (oblique wall condition); n = 4 * nseg_side * q.
// side of boundary node i: from the root box layout S (sx q), E (sy q), N (sx q), W (sy q).
// Block entry gi of the group: B = diag(nu) T_root + tau f G_t for pole alpha[gi].
__global__ void root_system(int nbatch, int n, int q, int sxq, int syq, const cd* __restrict__ alpha,
                            double tauf, const double* __restrict__ Ex, const double* __restrict__ Ey,
                            const cd* __restrict__ T, cd* B) {
  const size_t nn = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)nbatch * nn;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t gi = t / nn, e = t % nn;
    const cd al = alpha[gi];
    const int i = e % n, j = e / n;
    int side;
    if (i < sxq) side = 0;
    else if (i < sxq + syq) side = 1;
    else if (i < 2 * sxq + syq) side = 2;
    else side = 3;
    const double sg = (side == 1 || side == 2) ? 1.0 : -1.0;
    const cd tv = T[t];
    double re = sg * (al.x * tv.x - al.y * tv.y), im = sg * (al.x * tv.y + al.y * tv.x);
    // tangential derivative inside the same segment
    if (i / q == j / q) {
      const int a = i % q, c = j % q;
      if (side == 1 || side == 3) re += tauf * Ey[a * q + c];          // + tau f dh/dy on x-walls
      else re -= tauf * Ex[a * q + c];                                  // - tau f dh/dx on y-walls
    }
    B[t] = make_double2(re, im);
  }
}

// Root of a periodic square.  The root box's sides S and N are one seam (the same
// nodes, both in ascending x) and so are W and E (ascending y).  With the seam values
// s = [s_S (sxq); s_W (syq)] the boundary data are u_b = P s (u_S = u_N = s_S,
// u_W = u_E = s_W), and flux continuity across the seams (Section 2.2, the seams are
// interfaces between the last and the first leaf of a row or column) adds the outward
// fluxes of the two sides that meet there: P^T (T u_b + h) = 0.  So B = P^T T P
// (m x m, m = n / 2) and s = -B^{-1} P^T h.  B is column-major like T.
__device__ __forceinline__ void seam_pair(int r, int sxq, int syq, int& i1, int& i2) {
  if (r < sxq) { i1 = r; i2 = sxq + syq + r; }                      // S, N
  else { const int t = r - sxq; i1 = 2 * sxq + syq + t; i2 = sxq + t; }   // W, E
}

__global__ void root_periodic_system(int nbatch, int n, int sxq, int syq, const cd* __restrict__ T, cd* B) {
  const int m = n / 2;
  const size_t mm = (size_t)m * m, nn = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)nbatch * mm;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t gi = t / mm, e = t % mm;
    const int r = (int)(e % m), c = (int)(e / m);
    int i1, i2, j1, j2;
    seam_pair(r, sxq, syq, i1, i2);
    seam_pair(c, sxq, syq, j1, j2);
    const cd* Tg = T + gi * nn;
    const cd a = Tg[i1 + (size_t)j1 * n], b = Tg[i1 + (size_t)j2 * n];
    const cd d = Tg[i2 + (size_t)j1 * n], f = Tg[i2 + (size_t)j2 * n];
    B[t] = make_double2(a.x + b.x + d.x + f.x, a.y + b.y + d.y + f.y);
  }
}

// Fourier blocks of the rotation-symmetric wall system (square walled domain).  With
// the wall rows put in the rotation-covariant form (side k's rows times c4s(k)) and
// both rows and columns in counterclockwise side order, C_{k,l}[s][u] =
// c4s(k) B[idx_k(s)][idx_l(u)] is block circulant, C_{k,l} = c_{(l-k) mod 4}, and
// C y = r splits into the four systems Chat_m yhat_m = rhat_m, Chat_m = sum_d i^{md} c_d.
// c_d is the mean of C_{k,(k+d) mod 4} over the four k; the largest deviation of a
// C_{k,k+d} entry from it and the largest |B| entry go to stat[0..1] (atomic max of
// non-negative doubles through their bit patterns).  W: [nbatch][4][nq x nq],
// column-major like B.
__device__ __forceinline__ double c4s(int k) { return (k == 1 || k == 2) ? 1.0 : -1.0; }

__global__ void root_c4_blocks(int nbatch, int n, int nq, const int* __restrict__ idx, const cd* __restrict__ B,
                               cd* __restrict__ W, unsigned long long* stat) {
  const size_t per = (size_t)nq * nq;
  double dev = 0.0, bmax = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)nbatch * per;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t gi = t / per, e = t % per;
    const int sr = (int)(e % nq), u = (int)(e / nq);
    const cd* Bg = B + gi * (size_t)n * n;
    cd c[4];
    for (int d = 0; d < 4; ++d) {
      cd v[4];
      double mx = 0.0, my = 0.0;
      for (int k = 0; k < 4; ++k) {
        const cd b = Bg[idx[k * nq + sr] + (size_t)idx[((k + d) & 3) * nq + u] * n];
        v[k] = make_double2(c4s(k) * b.x, c4s(k) * b.y);
        mx += v[k].x;
        my += v[k].y;
        bmax = fmax(bmax, fmax(fabs(b.x), fabs(b.y)));
      }
      c[d] = make_double2(0.25 * mx, 0.25 * my);
      for (int k = 0; k < 4; ++k) dev = fmax(dev, fmax(fabs(v[k].x - c[d].x), fabs(v[k].y - c[d].y)));
    }
    for (int m = 0; m < 4; ++m) {
      double re = 0.0, im = 0.0;
      for (int d = 0; d < 4; ++d) {
        const cd x = c[d];
        switch ((m * d) & 3) {            // x * i^{md}
          case 0: re += x.x; im += x.y; break;
          case 1: re -= x.y; im += x.x; break;
          case 2: re -= x.x; im -= x.y; break;
          default: re += x.y; im -= x.x; break;
        }
      }
      W[(gi * 4 + m) * per + sr + (size_t)u * nq] = make_double2(re, im);
    }
  }
  atomicMax(&stat[0], (unsigned long long)__double_as_longlong(dev));
  atomicMax(&stat[1], (unsigned long long)__double_as_longlong(bmax));
}

// Even/odd blocks of a reflection-symmetric merge level (shared operators).  With Rb
// reversing the interface (t -> n3 - 1 - t) and the parent-boundary orbits mem[4 r + g]
// (g: 1, Ra, Rb, Ra Rb), for s, t < n3/2 and blk 0 (even, +) or 1 (odd, -):
//   Z rows:  ZUs[blk][s][t] = mean of ZU[s][t] +- ZU[s][Jt] and ZU[Js][Jt] +- ZU[Js][t],
//   U rows:  ZUs[blk][n3/2 + r][t] = mean over g of f_g (U[i_g][t] +- U[i_g][Jt]),
//   S:       Ss[blk][s][r] = mean over g of f_g (S[s][i_g] +- S[Js][i_g]) / 2,
// with f_g = -1 for the odd block on g = Rb, Ra Rb and +1 otherwise.  The largest
// deviation of one estimate from its mean and the largest |entry| read go to stat[0..1].
// ZU: [nbatch][zr x n3], S: [nbatch][n3 x nbd] column-major; ZUs [nbatch][2][rh x n3/2],
// Ss [nbatch][2][n3/2 x nbd/4].
__global__ void merge_sym_blocks(int nbatch, int n3, int nbd, int rh, int need_par, const int* __restrict__ mem,
                                 const cd* __restrict__ ZU, const cd* __restrict__ S, cd* __restrict__ ZUs,
                                 cd* __restrict__ Ss, unsigned long long* stat) {
  const int n3h = n3 / 2, nbq = need_par ? nbd / 4 : 0, zr = n3 + (need_par ? nbd : 0);
  const size_t zb = (size_t)rh * n3h, sb = (size_t)n3h * nbq;
  const size_t zper = 2 * zb, sper = 2 * sb, per = zper + sper;
  double dev = 0.0, amax = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)nbatch * per;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t gi = t / per, e = t % per;
    cd est[4];
    int ne = 0;
    if (e < zper) {
      const int blk = (int)(e / zb);
      const size_t f = e % zb;
      const int rho = (int)(f % rh), col = (int)(f / rh), tj = n3 - 1 - col;
      const double sg = blk ? -1.0 : 1.0;
      const cd* Zg = ZU + gi * (size_t)zr * n3;
      if (rho < n3h) {
        const int sr = rho, js = n3 - 1 - rho;
        const cd a = Zg[sr + (size_t)col * zr], b = Zg[sr + (size_t)tj * zr];
        const cd c = Zg[js + (size_t)tj * zr], d = Zg[js + (size_t)col * zr];
        est[0] = make_double2(a.x + sg * b.x, a.y + sg * b.y);
        est[1] = make_double2(c.x + sg * d.x, c.y + sg * d.y);
        ne = 2;
        amax = fmax(amax, fmax(fmax(fabs(a.x), fabs(a.y)), fmax(fabs(c.x), fabs(c.y))));
      } else {
        const int r = rho - n3h;
        for (int g = 0; g < 4; ++g) {
          const int i = mem[4 * r + g];
          const double fg = (blk && g >= 2) ? -1.0 : 1.0;
          const cd a = Zg[n3 + i + (size_t)col * zr], b = Zg[n3 + i + (size_t)tj * zr];
          est[g] = make_double2(fg * (a.x + sg * b.x), fg * (a.y + sg * b.y));
          amax = fmax(amax, fmax(fabs(a.x), fabs(a.y)));
        }
        ne = 4;
      }
      cd mean = make_double2(0.0, 0.0);
      for (int k = 0; k < ne; ++k) { mean.x += est[k].x / ne; mean.y += est[k].y / ne; }
      for (int k = 0; k < ne; ++k) dev = fmax(dev, fmax(fabs(est[k].x - mean.x), fabs(est[k].y - mean.y)));
      ZUs[gi * zper + blk * zb + rho + (size_t)col * rh] = mean;
    } else {
      const size_t e2 = e - zper;
      const int blk = (int)(e2 / sb);
      const size_t f = e2 % sb;
      const int sr = (int)(f % n3h), r = (int)(f / n3h), js = n3 - 1 - sr;
      const double sg = blk ? -1.0 : 1.0;
      const cd* Sg = S + gi * (size_t)n3 * nbd;
      cd mean = make_double2(0.0, 0.0);
      for (int g = 0; g < 4; ++g) {
        const int i = mem[4 * r + g];
        const double fg = (blk && g >= 2) ? -0.5 : 0.5;
        const cd a = Sg[sr + (size_t)i * n3], b = Sg[js + (size_t)i * n3];
        est[g] = make_double2(fg * (a.x + sg * b.x), fg * (a.y + sg * b.y));
        mean.x += 0.25 * est[g].x;
        mean.y += 0.25 * est[g].y;
        amax = fmax(amax, fmax(fabs(a.x), fabs(a.y)));
      }
      for (int g = 0; g < 4; ++g) dev = fmax(dev, fmax(fabs(est[g].x - mean.x), fabs(est[g].y - mean.y)));
      Ss[gi * sper + blk * sb + sr + (size_t)r * n3h] = mean;
    }
  }
  atomicMax(&stat[0], (unsigned long long)__double_as_longlong(dev));
  atomicMax(&stat[1], (unsigned long long)__double_as_longlong(amax));
}

namespace {

// Host-side fault injection for the error paths of the build (tests only):
// EO_FAULT_INJECT=singular makes the first leaf factorisation report a zero pivot
// (as cuBLAS getrf does for a singular block), EO_FAULT_INJECT=oom makes the first
// build workspace allocation fail.  Nothing is injected on the device.
int fault_inject() {
  const char* v = std::getenv("EO_FAULT_INJECT");
  if (!v) return 0;
  if (!std::strcmp(v, "singular")) return 1;
  if (!std::strcmp(v, "oom")) return 2;
  return 0;
}

struct Cublas {
  cublasHandle_t h = nullptr;
  ~Cublas() { if (h) cublasDestroy(h); }
};

// getrf + getrs(identity): Zout = inverse of each M (batched, in device memory).
eo_status batched_inverse(cublasHandle_t cb, cudaStream_t st, int n, int nbatch, cd* M, cd* Zout,
                          int* piv, int* info, std::vector<int>& hinfo, const char* what) {
  std::vector<cd*> pa(nbatch), pz(nbatch);
  for (int i = 0; i < nbatch; ++i) { pa[i] = M + (size_t)i * n * n; pz[i] = Zout + (size_t)i * n * n; }
  cd** dpa; cd** dpz;
  EO_CUDA_TRY(cudaMallocAsync(&dpa, sizeof(cd*) * nbatch, st));
  EO_CUDA_TRY(cudaMallocAsync(&dpz, sizeof(cd*) * nbatch, st));
  EO_CUDA_TRY(cudaMemcpyAsync(dpa, pa.data(), sizeof(cd*) * nbatch, cudaMemcpyHostToDevice, st));
  EO_CUDA_TRY(cudaMemcpyAsync(dpz, pz.data(), sizeof(cd*) * nbatch, cudaMemcpyHostToDevice, st));
  EO_CUBLAS_TRY(cublasZgetrfBatched(cb, n, (cuDoubleComplex**)dpa, n, piv, info, nbatch));
  hinfo.assign(nbatch, 0);
  EO_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * nbatch, cudaMemcpyDeviceToHost, st));
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < nbatch; ++i)
    if (hinfo[i] != 0) {
      cudaFreeAsync(dpa, st); cudaFreeAsync(dpz, st);
      return fail(EO_ERR_SINGULAR, std::string(what) + ": singular system (getrf info " +
                                       std::to_string(hinfo[i]) + ")");
    }
  set_identity<<<1024, 256, 0, st>>>(n, nbatch, Zout);
  int hi = 0;
  EO_CUBLAS_TRY(cublasZgetrsBatched(cb, CUBLAS_OP_N, n, n, (const cuDoubleComplex* const*)dpa, n, piv,
                                    (cuDoubleComplex* const*)dpz, n, &hi, nbatch));
  if (hi != 0) return fail(EO_ERR_INVALID_ARG, "getrs argument error");
  EO_CUDA_TRY(cudaFreeAsync(dpa, st));
  EO_CUDA_TRY(cudaFreeAsync(dpz, st));
  return EO_OK;
}

}  // namespace

eo_status build(Handle& h, const double* coeff, cudaStream_t st) {
  const Grid& g = h.g;
  const int p = g.p, q = g.q, ni = q * q, nb = 4 * q;
  const int nleaf = g.nlx * g.nly;
  const int nlo = h.shared ? 1 : nleaf;     // leaves with their own operators
  const int P = h.P;
  const int g_per = g.periodic;
  Cublas cbh;
  EO_CUBLAS_TRY(cublasCreate(&cbh.h));
  cublasHandle_t cb = cbh.h;
  EO_CUBLAS_TRY(cublasSetStream(cb, st));
  EO_CUBLAS_TRY(cublasSetPointerMode(cb, CUBLAS_POINTER_MODE_HOST));

  // scaled differentiation matrices on the device
  EO_CUDA_TRY(cudaMemcpyAsync(h.dDx, h.Dx, sizeof(double) * p * p, cudaMemcpyHostToDevice, st));
  EO_CUDA_TRY(cudaMemcpyAsync(h.dDx + p * p, h.Dy, sizeof(double) * p * p, cudaMemcpyHostToDevice, st));
  EO_CUDA_TRY(cudaMemcpyAsync(h.dDx + 2 * p * p, h.Ex, sizeof(double) * q * q, cudaMemcpyHostToDevice, st));
  EO_CUDA_TRY(cudaMemcpyAsync(h.dDx + 2 * p * p + q * q, h.Ey, sizeof(double) * q * q,
                              cudaMemcpyHostToDevice, st));
  const double* dDx = h.dDx;
  const double* dDy = h.dDx + p * p;
  const double* dEx = h.dDx + 2 * p * p;
  const double* dEy = dEx + q * q;

  // ---- leaf real matrices (pole independent)
  double *acoef = nullptr, *Aii0, *Aib, *Fbi, *Fbb;
  std::vector<void*> tmp;
  const int inject = fault_inject();
  auto talloc = [&](void** ptr, size_t bytes) -> eo_status {
    if (inject == 2) return fail(EO_ERR_OOM, "build workspace allocation failed (injected)");
    if (cudaMallocAsync(ptr, bytes, st) != cudaSuccess) return fail(EO_ERR_OOM, "build workspace allocation failed");
    tmp.push_back(*ptr);
    return EO_OK;
  };
  struct Freer {
    std::vector<void*>& v; cudaStream_t s;
    ~Freer() { for (void* x : v) cudaFreeAsync(x, s); cudaStreamSynchronize(s); }
  } freer{tmp, st};
  eo_status rc;
  if (h.kind == EO_WAVE_DIRICHLET) {
    acoef = h.acoef;   // kept: the apply's pre-map differentiates c^2 grad u
    EO_CUDA_TRY(cudaMemcpyAsync(acoef, coeff, sizeof(double) * g.n_nodes, cudaMemcpyHostToDevice, st));
  }
  if (h.kappa_form) {
    // 1 / kappa at every node: the shift's weight here, the source weight in the pre-map
    std::vector<double> w(g.n_nodes);
    for (int64_t i = 0; i < g.n_nodes; ++i) w[i] = 1.0 / coeff[i];
    EO_CUDA_TRY(cudaMemcpyAsync(h.hw, w.data(), sizeof(double) * g.n_nodes, cudaMemcpyHostToDevice, st));
    EO_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if ((rc = talloc((void**)&Aii0, sizeof(double) * nlo * ni * ni))) return rc;
  if ((rc = talloc((void**)&Aib, sizeof(double) * nlo * ni * nb))) return rc;
  if ((rc = talloc((void**)&Fbi, sizeof(double) * nlo * nb * ni))) return rc;
  if ((rc = talloc((void**)&Fbb, sizeof(double) * nlo * nb * nb))) return rc;
  EO_CUDA_TRY(cudaMemsetAsync(Aii0, 0, sizeof(double) * nlo * ni * ni, st));
  EO_CUDA_TRY(cudaMemsetAsync(Aib, 0, sizeof(double) * nlo * ni * nb, st));
  EO_CUDA_TRY(cudaMemsetAsync(Fbi, 0, sizeof(double) * nlo * nb * ni, st));
  EO_CUDA_TRY(cudaMemsetAsync(Fbb, 0, sizeof(double) * nlo * nb * nb, st));
  leaf_real_ops<<<nlo, 256, sizeof(double) * p * p, st>>>(g.nlx, g.nly, p, g.n_int, g.n_hseg, g.periodic, dDx,
                                                        dDy, acoef, Aii0, Aib, Fbi, Fbb);
  EO_CUDA_TRY(cudaGetLastError());
  if (h.fd && (rc = fd_setup(h, Aii0, Aib, Fbi, st))) return rc;
  // consistent shallow-water elimination: the leaf coupling of Curl(G h)
  double* Cib = nullptr;
  cd* dbeta = nullptr;
  if (h.kind == EO_SW_WALLS && h.opts.sw_consistent && h.opts.sw_f != 0.0) {
    if ((rc = talloc((void**)&Cib, sizeof(double) * nlo * ni * nb))) return rc;
    if ((rc = talloc((void**)&dbeta, sizeof(cd) * std::min(P, 64)))) return rc;
    leaf_curl_ops<<<nlo, 256, 0, st>>>(p, dDx, dDy, dEx, dEy, Cib);
    EO_CUDA_TRY(cudaGetLastError());
  }
  cd* Fbi_c;
  if ((rc = talloc((void**)&Fbi_c, sizeof(cd) * nlo * nb * ni))) return rc;
  real_to_complex<<<1024, 256, 0, st>>>((size_t)nlo * nb * ni, Fbi, Fbi_c);
  const Plan& plan = h.plan;
  const int L = plan.L();
  // Poles are processed in groups of G: with shared operators (one block per
  // level) a group batches many poles into each factorisation and product;
  // with per-box operators a single pole already batches every box.
  const int G = h.shared ? std::min(P, 64) : 1;
  size_t maxpiv = (size_t)G * nlo * ni, maxinfo = (size_t)G * nlo;
  size_t ws_merge = 0;   // complex entries for M33, Z, Q, Rm (or the root system)
  size_t maxT = (size_t)G * nlo * nb * nb;
  for (int l = 1; l <= L; ++l) {
    const Level& lv = plan.lv[l];
    const size_t nbo = (size_t)G * (h.shared ? 1 : lv.nbox);
    maxpiv = std::max(maxpiv, nbo * lv.n3);
    maxinfo = std::max(maxinfo, nbo);
    ws_merge = std::max(ws_merge, nbo * (2 * (size_t)lv.n3 * lv.n3 + 2 * (size_t)lv.nbd * lv.n3));
    maxT = std::max(maxT, nbo * lv.nbd * lv.nbd);
  }
  cd* c4w = nullptr;
  unsigned long long* c4stat = nullptr;
  unsigned long long* symstat = nullptr;
  if ((rc = talloc((void**)&symstat, sizeof(unsigned long long) * 2))) return rc;
  if (h.kind == EO_SW_WALLS || g_per) {
    maxpiv = std::max(maxpiv, (size_t)G * h.nroot);
    maxinfo = std::max(maxinfo, (size_t)G * (h.c4 ? 4 : 1));
    ws_merge = std::max(ws_merge, (size_t)G * h.nroot * h.nroot);
    if (h.c4) {
      if ((rc = talloc((void**)&c4w, sizeof(cd) * G * 4 * h.c4 * h.c4))) return rc;
      if ((rc = talloc((void**)&c4stat, sizeof(unsigned long long) * 2))) return rc;
    }
  }
  cd *Aw, *T0, *Tc, *Tn, *mw = nullptr, *kap, *dal;
  int *piv, *info;
  if ((rc = talloc((void**)&Aw, sizeof(cd) * G * nlo * ni * ni))) return rc;
  if ((rc = talloc((void**)&T0, sizeof(cd) * G * nlo * nb * nb))) return rc;
  if ((rc = talloc((void**)&Tc, sizeof(cd) * maxT))) return rc;
  if ((rc = talloc((void**)&Tn, sizeof(cd) * maxT))) return rc;
  if (ws_merge && (rc = talloc((void**)&mw, sizeof(cd) * ws_merge))) return rc;
  if ((rc = talloc((void**)&piv, sizeof(int) * maxpiv))) return rc;
  if ((rc = talloc((void**)&info, sizeof(int) * maxinfo))) return rc;
  if ((rc = talloc((void**)&kap, sizeof(cd) * G))) return rc;
  if ((rc = talloc((void**)&dal, sizeof(cd) * G))) return rc;
  std::vector<int> hinfo;
  const cuDoubleComplex one = {1.0, 0.0}, zero = {0.0, 0.0}, mone = {-1.0, 0.0};

  for (int p0 = 0; p0 < P; p0 += G) {
    const int g = std::min(G, P - p0);
    std::vector<cd> hk(g), ha(g);
    for (int gi = 0; gi < g; ++gi) {
      const std::complex<double> al = h.alpha[p0 + gi];
      const std::complex<double> k2 = kappa2(h, p0 + gi);
      hk[gi] = make_double2(k2.real(), k2.imag());
      ha[gi] = make_double2(al.real(), al.imag());
    }
    EO_CUDA_TRY(cudaMemcpyAsync(kap, hk.data(), sizeof(cd) * g, cudaMemcpyHostToDevice, st));
    EO_CUDA_TRY(cudaMemcpyAsync(dal, ha.data(), sizeof(cd) * g, cudaMemcpyHostToDevice, st));
    // ---- leaves: batch entries (pole of the group, leaf), contiguous blocks
    const int nbl = g * nlo;
    cd* XYp = h.XY + (size_t)p0 * h.xy_pstride;
    cd* Hp = h.H + (size_t)p0 * h.h_pstride;
    const long long xyb = (long long)ni * (ni + nb);
    const long long hb = (long long)nb * ni;
    if (Cib) {
      std::vector<cd> hb(g);
      for (int gi = 0; gi < g; ++gi) {
        const std::complex<double> bt = (h.tau * h.opts.sw_f) / h.alpha[p0 + gi];
        hb[gi] = make_double2(bt.real(), bt.imag());
      }
      EO_CUDA_TRY(cudaMemcpyAsync(dbeta, hb.data(), sizeof(cd) * g, cudaMemcpyHostToDevice, st));
    }
    leaf_assemble<<<2048, 256, 0, st>>>(nbl, nlo, ni, nb, kap, Aii0, Aib, Fbb, Cib, dbeta, h.hw, Aw, XYp, T0);
    EO_CUDA_TRY(cudaGetLastError());
    {
      std::vector<cd*> pa(nbl), pb(nbl);
      for (int i = 0; i < nbl; ++i) { pa[i] = Aw + (size_t)i * ni * ni; pb[i] = XYp + (size_t)i * xyb; }
      cd **dpa, **dpb;
      if ((rc = talloc((void**)&dpa, sizeof(cd*) * nbl))) return rc;
      if ((rc = talloc((void**)&dpb, sizeof(cd*) * nbl))) return rc;
      EO_CUDA_TRY(cudaMemcpyAsync(dpa, pa.data(), sizeof(cd*) * nbl, cudaMemcpyHostToDevice, st));
      EO_CUDA_TRY(cudaMemcpyAsync(dpb, pb.data(), sizeof(cd*) * nbl, cudaMemcpyHostToDevice, st));
      EO_CUBLAS_TRY(cublasZgetrfBatched(cb, ni, (cuDoubleComplex**)dpa, ni, piv, info, nbl));
      hinfo.assign(nbl, 0);
      EO_CUDA_TRY(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * nbl, cudaMemcpyDeviceToHost, st));
      EO_CUDA_TRY(cudaStreamSynchronize(st));
      if (inject == 1) hinfo[0] = 1;
      for (int i = 0; i < nbl; ++i)
        if (hinfo[i]) return fail(EO_ERR_SINGULAR, "leaf interior system singular (leaf " + std::to_string(i) + ")");
      int hi = 0;
      EO_CUBLAS_TRY(cublasZgetrsBatched(cb, CUBLAS_OP_N, ni, ni + nb, (const cuDoubleComplex* const*)dpa, ni, piv,
                                        (cuDoubleComplex* const*)dpb, ni, &hi, nbl));
      // T = Fbb + Fbi Y ; H = Fbi X  (Fbi per leaf; shared across the poles of a group)
      const long long fs = (G > 1) ? 0 : (long long)nb * ni;
      EO_CUBLAS_TRY(cublasZgemmStridedBatched(cb, CUBLAS_OP_N, CUBLAS_OP_N, nb, nb, ni, &one,
                                              (const cuDoubleComplex*)Fbi_c, nb, fs,
                                              (const cuDoubleComplex*)(XYp + (size_t)ni * ni), ni, xyb,
                                              &one, (cuDoubleComplex*)T0, nb, (long long)nb * nb, nbl));
      EO_CUBLAS_TRY(cublasZgemmStridedBatched(cb, CUBLAS_OP_N, CUBLAS_OP_N, nb, ni, ni, &one,
                                              (const cuDoubleComplex*)Fbi_c, nb, fs,
                                              (const cuDoubleComplex*)XYp, ni, xyb, &zero,
                                              (cuDoubleComplex*)Hp, nb, hb, nbl));
    }
    // ---- merges (parent T alternates between Tc and Tn; never the buffer being read)
    cd* Tprev = T0;
    int nbd_prev = nb, nbo_prev = nlo;
    for (int l = 1; l <= L; ++l) {
      const Level& lv = plan.lv[l];
      LevelDev& ld = h.lv[l];
      const int nbo = h.shared ? 1 : lv.nbox;
      const int nbt = g * nbo;   // batch entries at this level
      const int n3 = lv.n3, npar = lv.nbd;
      const bool root = (l == L);
      // a Dirichlet root keeps only Z; walls and periodic seams need the root's T
      const bool need_par = !(root && h.kind == EO_WAVE_DIRICHLET && !g_per);
      const bool need_T = !root || h.kind == EO_SW_WALLS || g_per;
      cd* M33 = mw;
      cd* Z = M33 + (size_t)nbt * n3 * n3;
      cd* Qm = Z + (size_t)nbt * n3 * n3;
      cd* Rm = Qm + (size_t)nbt * npar * n3;
      cd* Tw = (l % 2) ? Tc : Tn;
      merge_gather<<<nbt, 256, 0, st>>>(nbd_prev, n3, npar, ld.par_child, ld.par_idx, ld.a3, ld.b3, lv.dir,
                                        lv.nbx, plan.lv[l - 1].nbx, h.shared, nbo, nbo_prev, Tprev, M33,
                                        need_par ? Qm : nullptr, Rm, need_T ? Tw : nullptr);
      EO_CUDA_TRY(cudaGetLastError());
      if ((rc = batched_inverse(cb, st, n3, nbt, M33, Z, piv, info, hinfo, "merge interface system"))) return rc;
      cd* ZUp = ld.ZU + (size_t)p0 * ld.zu_pstride;
      const long long zub = (long long)ld.zu_rows * n3;
      copy_scaled<<<nbt, 256, 0, st>>>(n3, Z, ZUp, ld.zu_rows, zub, -1.0);
      if (need_par) {
        cd* Sp = ld.S + (size_t)p0 * ld.s_pstride;
        const long long sb = (long long)n3 * npar;
        // U = -Q Z  -> rows [n3, n3 + npar) of ZU
        EO_CUBLAS_TRY(cublasZgemmStridedBatched(cb, CUBLAS_OP_N, CUBLAS_OP_N, npar, n3, n3, &mone,
                                                (const cuDoubleComplex*)Qm, npar, (long long)npar * n3,
                                                (const cuDoubleComplex*)Z, n3, (long long)n3 * n3, &zero,
                                                (cuDoubleComplex*)(ZUp + n3), ld.zu_rows, zub, nbt));
        // S = -Z Rm
        EO_CUBLAS_TRY(cublasZgemmStridedBatched(cb, CUBLAS_OP_N, CUBLAS_OP_N, n3, npar, n3, &mone,
                                                (const cuDoubleComplex*)Z, n3, (long long)n3 * n3,
                                                (const cuDoubleComplex*)Rm, n3, (long long)n3 * npar, &zero,
                                                (cuDoubleComplex*)Sp, n3, sb, nbt));
        if (need_T) {
          // T_parent += Q S
          EO_CUBLAS_TRY(cublasZgemmStridedBatched(cb, CUBLAS_OP_N, CUBLAS_OP_N, npar, npar, n3, &one,
                                                  (const cuDoubleComplex*)Qm, npar, (long long)npar * n3,
                                                  (const cuDoubleComplex*)Sp, n3, sb, &one,
                                                  (cuDoubleComplex*)Tw, npar, (long long)npar * npar, nbt));
        }
      }
      if (ld.sym) {
        EO_CUDA_TRY(cudaMemsetAsync(symstat, 0, sizeof(unsigned long long) * 2, st));
        merge_sym_blocks<<<2048, 256, 0, st>>>(g, n3, npar, ld.rh, need_par ? 1 : 0, ld.mem, ZUp,
                                               need_par ? ld.S + (size_t)p0 * ld.s_pstride : nullptr,
                                               ld.ZUs + (size_t)p0 * ld.zs_pstride,
                                               ld.Ss ? ld.Ss + (size_t)p0 * ld.ss_pstride : nullptr, symstat);
        EO_CUDA_TRY(cudaGetLastError());
        unsigned long long hs[2];
        EO_CUDA_TRY(cudaMemcpyAsync(hs, symstat, sizeof(hs), cudaMemcpyDeviceToHost, st));
        EO_CUDA_TRY(cudaStreamSynchronize(st));
        double dev, amax;
        std::memcpy(&dev, &hs[0], sizeof(double));
        std::memcpy(&amax, &hs[1], sizeof(double));
        if (!(dev <= 1e-9 * amax))
          return fail(EO_ERR_UNSUPPORTED, "merge level " + std::to_string(l) +
                                              " is not reflection-symmetric (deviation " +
                                              std::to_string(dev / amax) + "); set opts.merge_dense");
      }
      Tprev = Tw;
      nbd_prev = npar;
      nbo_prev = nbo;
    }
    // ---- periodic seams: the root box merged with itself across both seams
    if (g_per) {
      const Level& rl = plan.lv[L];
      cd* Broot = mw;
      cd* Bi = h.Binv + (size_t)p0 * h.binv_pstride;
      root_periodic_system<<<2048, 256, 0, st>>>(g, rl.nbd, rl.sx * q, rl.sy * q, Tprev, Broot);
      EO_CUDA_TRY(cudaGetLastError());
      if ((rc = batched_inverse(cb, st, rl.nbd / 2, g, Broot, Bi, piv, info, hinfo, "periodic seam system")))
        return rc;
    } else if (h.kind == EO_SW_WALLS) {
      // ---- root oblique system (shallow-water walls)
      const Level& rl = plan.lv[L];
      const int n = rl.nbd;
      cd* Broot = mw;
      cd* Bi = h.Binv + (size_t)p0 * h.binv_pstride;
      root_system<<<2048, 256, 0, st>>>(g, n, q, rl.sx * q, rl.sy * q, dal, h.tau * h.opts.sw_f, dEx, dEy,
                                        Tprev, Broot);
      EO_CUDA_TRY(cudaGetLastError());
      if (h.c4) {
        const int nq = h.c4;
        EO_CUDA_TRY(cudaMemsetAsync(c4stat, 0, sizeof(unsigned long long) * 2, st));
        root_c4_blocks<<<2048, 256, 0, st>>>(g, n, nq, h.c4idx, Broot, c4w, c4stat);
        EO_CUDA_TRY(cudaGetLastError());
        unsigned long long hs[2];
        EO_CUDA_TRY(cudaMemcpyAsync(hs, c4stat, sizeof(hs), cudaMemcpyDeviceToHost, st));
        EO_CUDA_TRY(cudaStreamSynchronize(st));
        double dev, bmax;
        std::memcpy(&dev, &hs[0], sizeof(double));
        std::memcpy(&bmax, &hs[1], sizeof(double));
        if (!(dev <= 1e-9 * bmax))
          return fail(EO_ERR_UNSUPPORTED, "root wall system is not symmetric under the quarter turn (deviation " +
                                              std::to_string(dev / bmax) + "); set opts.root_dense");
        if ((rc = batched_inverse(cb, st, nq, 4 * g, c4w, Bi, piv, info, hinfo, "root wall Fourier block")))
          return rc;
      } else if ((rc = batched_inverse(cb, st, n, g, Broot, Bi, piv, info, hinfo, "root wall system"))) {
        return rc;
      }
    }
  }
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  h.aH = h.H;
  h.aXY = h.XY;
  h.aBinv = h.Binv;
  for (size_t l = 1; l < h.lv.size(); ++l) {
    h.lv[l].aZU = h.lv[l].ZU;
    h.lv[l].aS = h.lv[l].S;
    h.lv[l].aZUs = h.lv[l].ZUs;
    h.lv[l].aSs = h.lv[l].Ss;
  }
  return EO_OK;
}

// ---------------------------------------------------------------- reduced-precision copies
__global__ void to_float2(size_t n, const cd* __restrict__ x, float2* __restrict__ y) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = make_float2((float)x[t].x, (float)x[t].y);
}

// FP64 value -> (hi, lo) FP32 pair with hi = fl32(x), lo = fl32(x - hi)
__global__ void to_float_pair(size_t n, const cd* __restrict__ x, float4* __restrict__ y) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const cd v = x[t];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    y[t] = make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
  }
}

// Replace FP64 operator blocks by FP32 (prec 1) or FP32-pair (prec 2) copies.
// The top opts.fp64_top_levels merge levels (and then the root wall solve) keep
// FP64.  Vectors, pole sums and pre/post maps stay FP64 in every case.
eo_status to_reduced(Handle& h, int prec, cudaStream_t st) {
  auto conv = [&](cd*& src, size_t n, const void** view) -> eo_status {
    if (!src) { *view = nullptr; return EO_OK; }
    void* dst;
    const size_t esz = prec == 1 ? sizeof(float2) : sizeof(float4);
    eo_status rc = h.alloc(&dst, esz * n, true);
    if (rc) return rc;
    if (prec == 1) to_float2<<<4096, 256, 0, st>>>(n, src, (float2*)dst);
    else to_float_pair<<<4096, 256, 0, st>>>(n, src, (float4*)dst);
    EO_CUDA_TRY(cudaGetLastError());
    EO_CUDA_TRY(cudaStreamSynchronize(st));
    h.release(src, sizeof(cd) * n, true);
    src = nullptr;
    *view = dst;
    return EO_OK;
  };
  eo_status rc;
  const size_t P = h.P;
  if ((rc = conv(h.H, P * h.h_pstride, &h.aH))) return rc;
  if ((rc = conv(h.XY, P * h.xy_pstride, &h.aXY))) return rc;
  h.fp32 = prec;
  const int L = (int)h.lv.size() - 1;
  const int keep = std::max(0, h.opts.fp64_top_levels);
  for (int l = 1; l <= L - keep; ++l) {
    LevelDev& ld = h.lv[l];
    if ((rc = conv(ld.ZU, P * ld.zu_pstride, &ld.aZU))) return rc;
    if ((rc = conv(ld.S, P * ld.s_pstride, &ld.aS))) return rc;
    if ((rc = conv(ld.ZUs, P * ld.zs_pstride, &ld.aZUs))) return rc;
    if ((rc = conv(ld.Ss, P * ld.ss_pstride, &ld.aSs))) return rc;
    ld.fp32 = prec;
  }
  if (keep == 0) {
    if ((rc = conv(h.Binv, P * (size_t)h.binv_pstride, &h.aBinv))) return rc;
    h.root_fp32 = prec;
  }
  return EO_OK;
}

}  // namespace eo
