// Leaf level by fast diagonalisation (constant-coefficient leaves, shared
// per-level operators).
//
// On such a leaf the interior block of the collocated div(grad) (Section 2.2)
// is the Kronecker sum I (x) M_x + M_y (x) I, so for every pole
//     (A_ii - kappa_p^2)^{-1} = (V_y (x) V_x) diag(dinv_p) (V_y (x) V_x)^{-1},
//     dinv_p(a, b) = 1 / (lx_a + ly_b - kappa_p^2),
// and the boundary coupling A_ib and the flux rows F_bi are sums of outer
// products of 1-D vectors.  The two leaf stages of the apply (Section 2.3)
// then become, per pole and leaf, q-point transforms and a pointwise scaling:
//   up:   z^ = dinv_p * sum_k coef_pk g^_k (g^ = sources in the eigenbasis),
//         outward fluxes h_S = V_x (z^ rS^), h_N = V_x (z^ rN^),
//                        h_E = V_y (z^T rE^), h_W = V_y (z^T rW^);
//   down: the interior solution z_p = X g_p + Y u_b of Section 2.3 in the
//         eigenbasis is dinv_p * (g^_p - (A_ib u_b)^), with
//         (A_ib u_b)^(a, b) = cW^_a uW^_b + cE^_a uE^_b + uS^_a cS^_b + uN^_a cN^_b,
//         u^ the edge values in the 1-D eigenbases; the weighted pole sum of
//         the particular part, sum_p Re(w_pk coef_pk' dinv_p), does not depend
//         on the leaf and is formed once per call (gsum); each chunk of poles
//         maps its partial sum back with V_y (x) V_x.
// All of it is FP64.  Results equal the dense leaf operators up to rounding;
// the dense operators stay built for the adjoint sweeps.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sweep.cuh"

namespace eo {

// offsets (in doubles) inside the constant block h.fd_c
struct FdLayout {
  int q, qq;
  __host__ __device__ int Vx() const { return 0; }
  __host__ __device__ int Vxi() const { return qq; }
  __host__ __device__ int Vy() const { return 2 * qq; }
  __host__ __device__ int Vyi() const { return 3 * qq; }
  __host__ __device__ int lx() const { return 4 * qq; }
  __host__ __device__ int ly() const { return 4 * qq + q; }
  __host__ __device__ int cW() const { return 4 * qq + 2 * q; }
  __host__ __device__ int cE() const { return 4 * qq + 3 * q; }
  __host__ __device__ int cS() const { return 4 * qq + 4 * q; }
  __host__ __device__ int cN() const { return 4 * qq + 5 * q; }
  __host__ __device__ int rS() const { return 4 * qq + 6 * q; }
  __host__ __device__ int rN() const { return 4 * qq + 7 * q; }
  __host__ __device__ int rE() const { return 4 * qq + 8 * q; }
  __host__ __device__ int rW() const { return 4 * qq + 9 * q; }
  __host__ __device__ int size() const { return 4 * qq + 10 * q; }   // even
};

struct FdArgs {
  int q, K, ncol, nleaf;
  const double* c;       // constants, FdLayout (FP64)
  const double* gsum;    // [K][K][q*q] sum over the call's poles of Re(wgt[p][k] coef[p][k'] dinv_p)
  const double* ghat;    // [R][K][n_int] sources in the leaf eigenbasis
};

__host__ __device__ __forceinline__ size_t even_up(size_t n) { return (n + 1) & ~(size_t)1; }

// 16-byte asynchronous global -> shared copies (per-pole tables and edge values
// of the next pole are fetched while the current pole computes)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------- sources -> eigenbasis
// ghat[r][k][leaf](a, b) = sum_{k', j} Vxi[a][k'] Vyi[b][j] src_k(leaf, r)(k', j)
__global__ void __launch_bounds__(256) k_fd_src(Sweep s, FdArgs f, double* __restrict__ ghat) {
  extern __shared__ double fsm[];
  const int q = f.q, qq = q * q;
  const int box = blockIdx.x, r = blockIdx.y;
  const FdLayout Lo{q, qq};
  double* Vxi = fsm;
  double* Vyi = Vxi + qq;
  double* G = Vyi + qq;
  double* T = G + qq;
  for (int e = threadIdx.x; e < qq; e += blockDim.x) {
    Vxi[e] = f.c[Lo.Vxi() + e];
    Vyi[e] = f.c[Lo.Vyi() + e];
  }
  for (int kk = 0; kk < s.K; ++kk) {
    __syncthreads();
    for (int e = threadIdx.x; e < qq; e += blockDim.x)
      G[e] = s.src[kk][r * s.src_rs[kk] + (long long)box * qq + e];   // e = j q + k
    __syncthreads();
    for (int e = threadIdx.x; e < qq; e += blockDim.x) {
      const int a = e % q, j = e / q;
      double t = 0.0;
      for (int k = 0; k < q; ++k) t += Vxi[a * q + k] * G[j * q + k];
      T[j * q + a] = t;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < qq; e += blockDim.x) {
      const int a = e % q, b = e / q;
      double t = 0.0;
      for (int j = 0; j < q; ++j) t += T[j * q + a] * Vyi[b * q + j];
      ghat[((long long)(r * s.K + kk) * f.nleaf + box) * qq + e] = t;   // e = b q + a
    }
  }
}

// ---------------------------------------------------------------- arithmetic
// The leaf kernels are written once over an arithmetic policy:
//  - F64:  FP64 values and FMA accumulation (FP64 pipe);
//  - Pair: FP32 (hi, lo) pairs on the FP32 pipe: every product x*y of two
//          pairs is split exactly (p = fl(xh yh), e = fma(xh, yh, -p)) plus the
//          cross terms xh yl + xl yh, and accumulated with an error-free
//          two-sum into (s, c), c collecting the rounding errors and low parts
//          (~2^-48 relative, like the FP32-pair merge products).
// Shared-memory footprints are the same for both (8-byte reals, 16-byte complex).
struct F64 {
  typedef double R;
  typedef double A;
  typedef double2 CT;
  __device__ static R from(double x) { return x; }
  __device__ static double to(R x) { return x; }
  __device__ static A zero() { return 0.0; }
  __device__ static void mac(A& a, R x, R y) { a = fma(x, y, a); }
  __device__ static void msub(A& a, R x, R y) { a = fma(-x, y, a); }
  __device__ static R norm(A a) { return a; }
  __device__ static void acc_add(A& a, const A& b) { a += b; }
  __device__ static A acc_from(double v) { return v; }
  __device__ static double acc_to(A a) { return a; }
  __device__ static void ldc(const CT* p, R& re, R& im) { const CT v = __ldg(p); re = v.x; im = v.y; }
  __device__ static void lds(const CT* p, R& re, R& im) { const CT v = *p; re = v.x; im = v.y; }
  __device__ static CT mkc(double re, double im) { return make_double2(re, im); }
};

struct PairAcc { float s, c; };

struct Pair {
  typedef float2 R;      // (hi, lo)
  typedef PairAcc A;
  typedef float4 CT;     // (re hi, im hi, re lo, im lo)
  __device__ static R from(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
  }
  __device__ static double to(R x) { return (double)x.x + (double)x.y; }
  __device__ static A zero() { return PairAcc{0.f, 0.f}; }
  __device__ static void acc_prod(A& a, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    const float e = __fmaf_rn(xh, yh, -p);
    const float lo = __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, e));
    const float t = __fadd_rn(a.s, p);
    const float bp = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, __fadd_rn(err, lo));
  }
  __device__ static void mac(A& a, R x, R y) { acc_prod(a, x.x, x.y, y.x, y.y); }
  __device__ static void msub(A& a, R x, R y) { acc_prod(a, -x.x, -x.y, y.x, y.y); }
  __device__ static R norm(A a) {
    const float h = __fadd_rn(a.s, a.c);
    return make_float2(h, __fsub_rn(a.c, __fsub_rn(h, a.s)));
  }
  __device__ static A acc_from(double v) {
    const float h = __double2float_rn(v);
    return PairAcc{h, __double2float_rn(v - (double)h)};
  }
  // a += b for two accumulators: two-sum of the leading parts, corrections added
  __device__ static void acc_add(A& a, const A& b) {
    const float t = __fadd_rn(a.s, b.s);
    const float bp = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(b.s, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, __fadd_rn(b.c, err));
  }
  __device__ static double acc_to(A a) { return (double)a.s + (double)a.c; }
  __device__ static void ldc(const CT* p, R& re, R& im) {
    const CT v = __ldg(p);
    re = make_float2(v.x, v.z);
    im = make_float2(v.y, v.w);
  }
  __device__ static void lds(const CT* p, R& re, R& im) {
    const CT v = *p;
    re = make_float2(v.x, v.z);
    im = make_float2(v.y, v.w);
  }
  __device__ static CT mkc(double re, double im) {
    const float rh = __double2float_rn(re), ih = __double2float_rn(im);
    return make_float4(rh, ih, __double2float_rn(re - (double)rh), __double2float_rn(im - (double)ih));
  }
};

template <class M>
struct Cx { typename M::R re, im; };

// FP64 constants (FdLayout) -> the policy's reals
template <class M>
__device__ __forceinline__ void load_consts(const double* c, typename M::R* cst, int n) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) cst[e] = M::from(c[e]);
}

// ---------------------------------------------------------------- up: leaf fluxes
// Block: ncol columns (leaf, rhs) x q threads; thread (c, a) owns eigen row a of
// column c.  Blocks along y take consecutive chunks of ppc poles.
// QR > 0: q == QR and K == 3 fixed at compile time; each thread keeps its row of
// the transformed sources g^ in registers (no shared copy).  QR == 0: any q.
template <class M, int QR>
__global__ void __launch_bounds__(256) k_fd_up_leaf(Sweep s, FdArgs f, const typename M::CT* __restrict__ dct,
                                                    int ppc, cd* __restrict__ h0) {
  typedef typename M::R R;
  typedef typename M::A A;
  extern __shared__ double fsm[];
  constexpr bool REG = QR > 0;
  const int q = REG ? QR : f.q, qq = q * q, K = REG ? 3 : s.K, ncol = f.ncol;
  const FdLayout Lo{q, qq};
  const int c = threadIdx.x / q, a = threadIdx.x - c * q;
  const int ncols = f.nleaf * s.R;
  const int col = blockIdx.x * ncol + c;
  const bool valid = col < ncols;
  int box = 0, r = 0;
  if (valid) col_box(col, s.R, box, r);
  R* cst = (R*)fsm;
  R* gs = cst + Lo.size();
  Cx<M>* zs = (Cx<M>*)(gs + (REG ? 0 : even_up((size_t)ncol * K * qq)));
  Cx<M>* ts = zs + (size_t)ncol * qq;   // [2][ncol][4][q]
  typename M::CT* dcs = (typename M::CT*)(ts + (size_t)2 * ncol * 4 * q);   // [2][K][qq] pole tables
  R gr[REG ? 3 : 1][REG ? QR : 1];
  load_consts<M>(f.c, cst, Lo.size());
  if constexpr (REG) {
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
      for (int bq = 0; bq < QR; ++bq)
        gr[kk][bq] = M::from(valid ? f.ghat[((long long)(r * 3 + kk) * f.nleaf + box) * qq + bq * QR + a] : 0.0);
  } else {
    for (int e = threadIdx.x; e < ncol * K * qq; e += blockDim.x) {
      const int cc = e / (K * qq), rem = e - cc * K * qq, kk = rem / qq, idx = rem - kk * qq;
      const int colc = blockIdx.x * ncol + cc;
      double v = 0.0;
      if (colc < ncols) {
        int bx, rr;
        col_box(colc, s.R, bx, rr);
        v = f.ghat[((long long)(rr * K + kk) * f.nleaf + bx) * qq + idx];
      }
      gs[e] = M::from(v);
    }
  }
  __syncthreads();
  const R* Vx = cst + Lo.Vx();
  const R* Vy = cst + Lo.Vy();
  const R* rS = cst + Lo.rS();
  const R* rN = cst + Lo.rN();
  const R* rE = cst + Lo.rE();
  const R* rW = cst + Lo.rW();
  const R* g = gs + (size_t)c * K * qq;   // shared variant only
  Cx<M>* zc = zs + (size_t)c * qq;
  const int pbeg = blockIdx.y * ppc, pend = min(s.P, pbeg + ppc);
  auto prefetch = [&](int pl, int bf) {
    const typename M::CT* src = dct + (size_t)(s.p0 + pl) * K * qq;
    typename M::CT* dst = dcs + (size_t)bf * K * qq;
    for (int e = threadIdx.x; e < K * qq; e += blockDim.x) cp_async16(dst + e, src + e);
    cp_async_commit();
  };
  if (pbeg < pend) prefetch(pbeg, 0);
  int buf = 0;
  for (int pl = pbeg; pl < pend; ++pl) {
    // this pole's table has landed; every thread is past the previous pole,
    // so the other buffer can take the next pole's table
    cp_async_wait_all();
    __syncthreads();
    if (pl + 1 < pend) prefetch(pl + 1, buf ^ 1);
    const typename M::CT* DC = dcs + (size_t)buf * K * qq;
    Cx<M>* tb = ts + (size_t)(buf * ncol + c) * 4 * q;
    // z^(a, b) = sum_k dc_k(a, b) g^_k(a, b); row contractions with rS^, rN^.
    // Two columns b, b + 1 per iteration with separate partial sums (more
    // independent dependency chains per thread).
    A sr[2], si[2], nr[2], ni_[2];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) sr[h2] = si[h2] = nr[h2] = ni_[h2] = M::zero();
    int b = 0;
    if constexpr (REG) {
#pragma unroll
      for (int bq = 0; bq < QR; ++bq) {
        const int idx = bq * QR + a, h2 = bq & 1;
        A zr = M::zero(), zi = M::zero();
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          R dr, di;
          M::lds(DC + kk * qq + idx, dr, di);
          M::mac(zr, dr, gr[kk][bq]);
          M::mac(zi, di, gr[kk][bq]);
        }
        const R zre = M::norm(zr), zim = M::norm(zi);
        M::mac(sr[h2], zre, rS[bq]); M::mac(si[h2], zim, rS[bq]);
        M::mac(nr[h2], zre, rN[bq]); M::mac(ni_[h2], zim, rN[bq]);
        zc[idx] = Cx<M>{zre, zim};
      }
      b = q;
    }
    for (; b + 1 < q; b += 2) {
      const int i0 = b * q + a, i1 = i0 + q;
      A zr0 = M::zero(), zi0 = M::zero(), zr1 = M::zero(), zi1 = M::zero();
      for (int kk = 0; kk < K; ++kk) {
        R dr0, di0, dr1, di1;
        M::lds(DC + kk * qq + i0, dr0, di0);
        M::lds(DC + kk * qq + i1, dr1, di1);
        const R g0 = g[kk * qq + i0], g1 = g[kk * qq + i1];
        M::mac(zr0, dr0, g0); M::mac(zi0, di0, g0);
        M::mac(zr1, dr1, g1); M::mac(zi1, di1, g1);
      }
      const R zre0 = M::norm(zr0), zim0 = M::norm(zi0), zre1 = M::norm(zr1), zim1 = M::norm(zi1);
      M::mac(sr[0], zre0, rS[b]); M::mac(si[0], zim0, rS[b]);
      M::mac(nr[0], zre0, rN[b]); M::mac(ni_[0], zim0, rN[b]);
      M::mac(sr[1], zre1, rS[b + 1]); M::mac(si[1], zim1, rS[b + 1]);
      M::mac(nr[1], zre1, rN[b + 1]); M::mac(ni_[1], zim1, rN[b + 1]);
      zc[i0] = Cx<M>{zre0, zim0};
      zc[i1] = Cx<M>{zre1, zim1};
    }
    if (b < q) {
      const int idx = b * q + a;
      A zr = M::zero(), zi = M::zero();
      for (int kk = 0; kk < K; ++kk) {
        R dr, di;
        M::lds(DC + kk * qq + idx, dr, di);
        const R gv = g[kk * qq + idx];
        M::mac(zr, dr, gv);
        M::mac(zi, di, gv);
      }
      const R zre = M::norm(zr), zim = M::norm(zi);
      M::mac(sr[0], zre, rS[b]); M::mac(si[0], zim, rS[b]);
      M::mac(nr[0], zre, rN[b]); M::mac(ni_[0], zim, rN[b]);
      zc[idx] = Cx<M>{zre, zim};
    }
    M::acc_add(sr[0], sr[1]); M::acc_add(si[0], si[1]);
    M::acc_add(nr[0], nr[1]); M::acc_add(ni_[0], ni_[1]);
    tb[a] = Cx<M>{M::norm(sr[0]), M::norm(si[0])};
    tb[2 * q + a] = Cx<M>{M::norm(nr[0]), M::norm(ni_[0])};
    __syncthreads();
    // column contractions with rE^, rW^ (thread a takes column b = a)
    {
      A er[2], ei[2], wr[2], wi[2];
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) er[h2] = ei[h2] = wr[h2] = wi[h2] = M::zero();
      int m = 0;
      for (; m + 1 < q; m += 2) {
        const Cx<M> z0 = zc[a * q + m], z1 = zc[a * q + m + 1];
        M::mac(er[0], z0.re, rE[m]); M::mac(ei[0], z0.im, rE[m]);
        M::mac(wr[0], z0.re, rW[m]); M::mac(wi[0], z0.im, rW[m]);
        M::mac(er[1], z1.re, rE[m + 1]); M::mac(ei[1], z1.im, rE[m + 1]);
        M::mac(wr[1], z1.re, rW[m + 1]); M::mac(wi[1], z1.im, rW[m + 1]);
      }
      if (m < q) {
        const Cx<M> z = zc[a * q + m];
        M::mac(er[0], z.re, rE[m]); M::mac(ei[0], z.im, rE[m]);
        M::mac(wr[0], z.re, rW[m]); M::mac(wi[0], z.im, rW[m]);
      }
      M::acc_add(er[0], er[1]); M::acc_add(ei[0], ei[1]);
      M::acc_add(wr[0], wr[1]); M::acc_add(wi[0], wi[1]);
      tb[q + a] = Cx<M>{M::norm(er[0]), M::norm(ei[0])};
      tb[3 * q + a] = Cx<M>{M::norm(wr[0]), M::norm(wi[0])};
    }
    __syncthreads();
    // back to nodal edge values: h_S, h_N through V_x; h_E, h_W through V_y
    if (valid) {
      A hs[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) hs[i] = M::zero();
      for (int m = 0; m < q; ++m) {
        const R vx = Vx[a * q + m], vy = Vy[a * q + m];
        const Cx<M> t0 = tb[m], t1 = tb[q + m], t2 = tb[2 * q + m], t3 = tb[3 * q + m];
        M::mac(hs[0], vx, t0.re); M::mac(hs[1], vx, t0.im);
        M::mac(hs[2], vy, t1.re); M::mac(hs[3], vy, t1.im);
        M::mac(hs[4], vx, t2.re); M::mac(hs[5], vx, t2.im);
        M::mac(hs[6], vy, t3.re); M::mac(hs[7], vy, t3.im);
      }
      cd* out = h0 + (((size_t)pl * s.R + r) * f.nleaf + box) * s.nb;
      out[a] = make_double2(M::acc_to(hs[0]), M::acc_to(hs[1]));           // S
      out[q + a] = make_double2(M::acc_to(hs[2]), M::acc_to(hs[3]));       // E
      out[2 * q + a] = make_double2(M::acc_to(hs[4]), M::acc_to(hs[5]));   // N
      out[3 * q + a] = make_double2(M::acc_to(hs[6]), M::acc_to(hs[7]));   // W
    }
    buf ^= 1;
  }
}

// ---------------------------------------------------------------- down: leaf interiors + pole sum
// QR > 0: q == QR and K == 3 fixed at compile time; each thread keeps its row of
// the pole-sum accumulators in registers (no shared-memory read-modify-write,
// smaller shared footprint, more resident blocks).  QR == 0: any q, accumulators
// in shared memory.
template <class M, int QR>
__global__ void __launch_bounds__(256) k_fd_down_leaf(Sweep s, FdArgs f, const typename M::CT* __restrict__ wdt,
                                                      const int* __restrict__ bseg, int ppc,
                                                      const cd* __restrict__ E, double* __restrict__ part) {
  typedef typename M::R R;
  typedef typename M::A A;
  extern __shared__ double fsm[];
  constexpr bool REG = QR > 0;
  const int q = REG ? QR : f.q, qq = q * q, K = REG ? 3 : s.K, ncol = f.ncol;
  const FdLayout Lo{q, qq};
  const int c = threadIdx.x / q, a = threadIdx.x - c * q;
  const int ncols = f.nleaf * s.R;
  const int col = blockIdx.x * ncol + c;
  const bool valid = col < ncols;
  const int chunk = blockIdx.y;
  int box = 0, r = 0;
  if (valid) col_box(col, s.R, box, r);
  R* cst = (R*)fsm;
  A* acc = (A*)(cst + Lo.size());                                  // [ncol][K][qq] (shared variant)
  R* T = REG ? (R*)(cst + Lo.size()) : (R*)(acc + even_up((size_t)ncol * K * qq));   // [ncol][qq]
  A accr[REG ? 3 : 1][REG ? QR : 1];                               // register variant
  Cx<M>* ub = (Cx<M>*)(T + even_up((size_t)ncol * qq));            // [ncol][4][q]
  Cx<M>* uh = ub + (size_t)ncol * 4 * q;                           // [ncol][4][q]
  typename M::CT* wds = (typename M::CT*)(uh + (size_t)ncol * 4 * q);   // [2][K][qq] pole tables
  cd* rb = (cd*)(wds + (size_t)2 * K * qq);                        // [2][ncol][4][q] raw edge values
  load_consts<M>(f.c, cst, Lo.size());
  // chunk 0 starts from the pole-summed particular part, sum_k' gsum[k][k'] g^_k'
  if constexpr (REG) {
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
      for (int bq = 0; bq < QR; ++bq) {
        double v = 0.0;
        const int idx = bq * QR + a;
        if (chunk == 0 && valid)
          for (int k2 = 0; k2 < 3; ++k2)
            v = fma(f.gsum[(kk * 3 + k2) * qq + idx], f.ghat[((long long)(r * 3 + k2) * f.nleaf + box) * qq + idx], v);
        accr[kk][bq] = M::acc_from(v);
      }
  } else {
    for (int e = threadIdx.x; e < ncol * K * qq; e += blockDim.x) {
      const int cc = e / (K * qq), rem = e - cc * K * qq, kk = rem / qq, idx = rem - kk * qq;
      const int colc = blockIdx.x * ncol + cc;
      double v = 0.0;
      if (chunk == 0 && colc < ncols) {
        int bx, rr;
        col_box(colc, s.R, bx, rr);
        for (int k2 = 0; k2 < K; ++k2)
          v = fma(f.gsum[(kk * K + k2) * qq + idx], f.ghat[((long long)(rr * K + k2) * f.nleaf + bx) * qq + idx], v);
      }
      acc[e] = M::acc_from(v);
    }
  }
  const R* Vxi = cst + Lo.Vxi();
  const R* Vyi = cst + Lo.Vyi();
  const R* cS = cst + Lo.cS();
  const R* cN = cst + Lo.cN();
  const R cWa = M::from(f.c[Lo.cW() + a]), cEa = M::from(f.c[Lo.cE() + a]);
  Cx<M>* ubc = ub + (size_t)c * 4 * q;
  Cx<M>* uhc = uh + (size_t)c * 4 * q;
  A* ac = acc + (size_t)c * K * qq;
  const int pbeg = chunk * ppc, pend = min(s.P, pbeg + ppc);
  auto prefetch = [&](int pl, int bf) {
    const typename M::CT* src = wdt + (size_t)pl * K * qq;
    typename M::CT* dst = wds + (size_t)bf * K * qq;
    for (int e = threadIdx.x; e < K * qq; e += blockDim.x) cp_async16(dst + e, src + e);
    if (valid) {
      const cd* Ep = E + ((size_t)pl * s.R + r) * s.n_edge;
      cd* rbc = rb + ((size_t)bf * ncol + c) * 4 * q;
      for (int side = 0; side < 4; ++side) cp_async16(rbc + side * q + a, Ep + (size_t)bseg[box * 4 + side] * q + a);
    }
    cp_async_commit();
  };
  if (pbeg < pend) prefetch(pbeg, 0);
  for (int pl = pbeg; pl < pend; ++pl) {
    const int buf = (pl - pbeg) & 1;
    // this pole's edge values and weights have landed; every thread is past
    // the previous pole, so the other buffers can take the next pole's
    cp_async_wait_all();
    __syncthreads();
    if (pl + 1 < pend) prefetch(pl + 1, buf ^ 1);
    // edge values of this leaf, sides S, E, N, W
    const cd* rbc = rb + ((size_t)buf * ncol + c) * 4 * q;
    for (int side = 0; side < 4; ++side) {
      const cd u = valid ? rbc[side * q + a] : make_double2(0.0, 0.0);
      ubc[side * q + a] = Cx<M>{M::from(u.x), M::from(u.y)};
    }
    __syncthreads();
    // to the 1-D eigenbases: S, N along x (Vxi); E, W along y (Vyi)
    {
      A v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = M::zero();
      for (int m = 0; m < q; ++m) {
        const R vx = Vxi[a * q + m], vy = Vyi[a * q + m];
        const Cx<M> u0 = ubc[m], u1 = ubc[q + m], u2 = ubc[2 * q + m], u3 = ubc[3 * q + m];
        M::mac(v[0], vx, u0.re); M::mac(v[1], vx, u0.im);
        M::mac(v[2], vy, u1.re); M::mac(v[3], vy, u1.im);
        M::mac(v[4], vx, u2.re); M::mac(v[5], vx, u2.im);
        M::mac(v[6], vy, u3.re); M::mac(v[7], vy, u3.im);
      }
      uhc[a] = Cx<M>{M::norm(v[0]), M::norm(v[1])};
      uhc[q + a] = Cx<M>{M::norm(v[2]), M::norm(v[3])};
      uhc[2 * q + a] = Cx<M>{M::norm(v[4]), M::norm(v[5])};
      uhc[3 * q + a] = Cx<M>{M::norm(v[6]), M::norm(v[7])};
    }
    __syncthreads();
    // acc_k(a, b) -= Re(wd_k(a, b) (A_ib u_b)^(a, b))
    const Cx<M> uSa = uhc[a], uNa = uhc[2 * q + a];
    const typename M::CT* W = wds + (size_t)buf * K * qq;
    // (A_ib u_b)^(a, b) for one column b, then the weighted update of acc
    auto bnd = [&](int b, R& brn, R& bin) {
      const Cx<M> uE = uhc[q + b], uW = uhc[3 * q + b];
      const R cs = cS[b], cn = cN[b];
      A br = M::zero(), bi = M::zero();
      M::mac(br, cWa, uW.re); M::mac(bi, cWa, uW.im);
      M::mac(br, cEa, uE.re); M::mac(bi, cEa, uE.im);
      M::mac(br, uSa.re, cs); M::mac(bi, uSa.im, cs);
      M::mac(br, uNa.re, cn); M::mac(bi, uNa.im, cn);
      brn = M::norm(br);
      bin = M::norm(bi);
    };
    if constexpr (REG) {
#pragma unroll
      for (int bq = 0; bq < QR; ++bq) {
        const int idx = bq * QR + a;
        R brn, bin;
        bnd(bq, brn, bin);
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          R wr, wi;
          M::lds(W + kk * qq + idx, wr, wi);
          M::msub(accr[kk][bq], wr, brn);
          M::mac(accr[kk][bq], wi, bin);
        }
      }
      continue;
    }
    int b = 0;
    for (; b + 1 < q; b += 2) {
      const int i0 = b * q + a, i1 = i0 + q;
      R br0, bi0, br1, bi1;
      bnd(b, br0, bi0);
      bnd(b + 1, br1, bi1);
      for (int kk = 0; kk < K; ++kk) {
        R wr0, wi0, wr1, wi1;
        M::lds(W + kk * qq + i0, wr0, wi0);
        M::lds(W + kk * qq + i1, wr1, wi1);
        A t0 = ac[kk * qq + i0], t1 = ac[kk * qq + i1];
        M::msub(t0, wr0, br0); M::mac(t0, wi0, bi0);
        M::msub(t1, wr1, br1); M::mac(t1, wi1, bi1);
        ac[kk * qq + i0] = t0;
        ac[kk * qq + i1] = t1;
      }
    }
    if (b < q) {
      const int idx = b * q + a;
      R brn, bin;
      bnd(b, brn, bin);
      for (int kk = 0; kk < K; ++kk) {
        R wr, wi;
        M::lds(W + kk * qq + idx, wr, wi);
        A t = ac[kk * qq + idx];
        M::msub(t, wr, brn);
        M::mac(t, wi, bin);
        ac[kk * qq + idx] = t;
      }
    }
  }
  // partial sums back to nodal values: Z = V_x acc V_y^T
  const R* Vx = cst + Lo.Vx();
  const R* Vy = cst + Lo.Vy();
  R* Tc = T + (size_t)c * qq;
  for (int kk = 0; kk < K; ++kk) {
    __syncthreads();
    if constexpr (REG) {
      R an[QR];
#pragma unroll
      for (int bq = 0; bq < QR; ++bq) {
        A v = accr[0][bq];
        if (kk == 1) v = accr[1][bq];
        if (kk == 2) v = accr[2][bq];
        an[bq] = M::norm(v);
      }
      for (int j = 0; j < q; ++j) {
        A t = M::zero();
#pragma unroll
        for (int bq = 0; bq < QR; ++bq) M::mac(t, an[bq], Vy[j * q + bq]);
        Tc[j * q + a] = M::norm(t);
      }
    } else {
      const A* ak = ac + kk * qq;
      for (int j = 0; j < q; ++j) {
        A t = M::zero();
        for (int b = 0; b < q; ++b) M::mac(t, M::norm(ak[b * q + a]), Vy[j * q + b]);
        Tc[j * q + a] = M::norm(t);
      }
    }
    __syncthreads();
    if (valid) {
      double* out = part + (((size_t)chunk * s.R + r) * K + kk) * s.n_int + (size_t)box * qq;
      for (int j = 0; j < q; ++j) {
        A z = M::zero();
        for (int m = 0; m < q; ++m) M::mac(z, Vx[a * q + m], Tc[j * q + m]);
        out[j * q + a] = M::acc_to(z);
      }
    }
  }
}

// ---------------------------------------------------------------- per-call tables
// wd[pl][k] = wgt[p0 + pl][k] * dinv_p (FP64 product, stored in the policy's format)
template <class M>
__global__ void k_fd_wd(int np, int p0, int K, int qq, const cd* __restrict__ wgt, const cd* __restrict__ dinv,
                        typename M::CT* __restrict__ wd) {
  const size_t tot = (size_t)np * K * qq;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int pl = (int)(t / ((size_t)K * qq));
    const int rem = (int)(t - (size_t)pl * K * qq), kk = rem / qq, idx = rem - kk * qq;
    const cd w = wgt[(p0 + pl) * K + kk], d = dinv[(size_t)(p0 + pl) * qq + idx];
    wd[t] = M::mkc(w.x * d.x - w.y * d.y, w.x * d.y + w.y * d.x);
  }
}

// gsum[k][k'](a, b) = sum_p Re(wgt[p][k] coef[p][k'] dinv_p(a, b)).  A block takes
// 32 consecutive outputs; its 32 warps stride over the poles and the warp
// partials are added in a fixed order (deterministic).
__global__ void __launch_bounds__(1024) k_fd_gsum(int np, int p0, int K, int qq, const cd* __restrict__ wgt,
                                                  const cd* __restrict__ coef, const cd* __restrict__ dinv,
                                                  double* __restrict__ gsum) {
  __shared__ double red[32][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  const bool ok = t < K * K * qq;
  const int kk = ok ? t / (K * qq) : 0, k2 = ok ? (t / qq) % K : 0, idx = ok ? t % qq : 0;
  double sum = 0.0;
  if (ok)
    for (int pl = wp; pl < np; pl += 32) {
      const int p = p0 + pl;
      const cd w = wgt[p * K + kk], cf = coef[p * K + k2], d = dinv[(size_t)p * qq + idx];
      const double wr = w.x * cf.x - w.y * cf.y, wi = w.x * cf.y + w.y * cf.x;
      sum = fma(wr, d.x, fma(-wi, d.y, sum));
    }
  red[wp][lane] = sum;
  __syncthreads();
  if (wp == 0 && ok) {
    double v = 0.0;
    for (int w = 0; w < 32; ++w) v += red[w][lane];
    gsum[t] = v;
  }
}

// dc[p][k] = coef[p][k] * dinv_p (build time)
template <class M>
__global__ void k_fd_dc(int P, int K, int qq, const cd* __restrict__ coef, const cd* __restrict__ dinv,
                        typename M::CT* __restrict__ dc) {
  const size_t tot = (size_t)P * K * qq;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(t / ((size_t)K * qq));
    const int rem = (int)(t - (size_t)p * K * qq), kk = rem / qq, idx = rem - kk * qq;
    const cd w = coef[p * K + kk], d = dinv[(size_t)p * qq + idx];
    dc[t] = M::mkc(w.x * d.x - w.y * d.y, w.x * d.y + w.y * d.x);
  }
}

namespace {

int fd_ncol(int q, int tuned) { return tuned > 0 ? tuned : std::max(1, 128 / q); }

FdArgs fd_args(const Handle& h, int nleaf, int ncol) {
  FdArgs f;
  f.q = h.g.q; f.K = h.K; f.ncol = fd_ncol(h.g.q, ncol); f.nleaf = nleaf;
  f.c = h.fd_c; f.gsum = h.fd_gsum; f.ghat = h.fd_ghat;
  return f;
}

// leaf q with register instantiations of the leaf kernels (K = 3)
constexpr int kFdRegQ = 14;
bool fd_down_reg(int q, int K) { return q == kFdRegQ && K == 3; }

size_t fd_up_smem(int q, int K, int ncol) {
  const int qq = q * q;
  const size_t gsd = fd_down_reg(q, K) ? 0 : even_up((size_t)ncol * K * qq);
  return sizeof(double) * ((size_t)4 * qq + 10 * q + gsd) +
         sizeof(cd) * ((size_t)ncol * qq + (size_t)2 * ncol * 4 * q + (size_t)2 * K * qq);
}


size_t fd_down_smem(int q, int K, int ncol) {
  const int qq = q * q;
  const size_t accd = fd_down_reg(q, K) ? 0 : even_up((size_t)ncol * K * qq);
  return sizeof(double) * ((size_t)4 * qq + 10 * q + accd + even_up((size_t)ncol * qq)) +
         sizeof(cd) * ((size_t)2 * ncol * 4 * q + (size_t)2 * K * qq + (size_t)2 * ncol * 4 * q);
}

template <class M>
eo_status up_leaf_t(Handle& h, const Sweep& s, const FdArgs& f, cd* h0, cudaStream_t st) {
  const int q = f.q;
  const int ncols = f.nleaf * s.R;
  const int ngroups = (ncols + f.ncol - 1) / f.ncol;
  int nchunk = std::max(1, std::min(s.P, (608 + ngroups - 1) / ngroups));
  const int ppc = (s.P + nchunk - 1) / nchunk;
  nchunk = (s.P + ppc - 1) / ppc;
  const size_t smem = fd_up_smem(q, s.K, f.ncol);
  const typename M::CT* dct = (const typename M::CT*)h.fd_dc;
  if (fd_down_reg(q, s.K)) {
    static size_t cap[64] = {};
    eo_status rc = ensure_smem((const void*)k_fd_up_leaf<M, kFdRegQ>, smem, cap, 0);
    if (rc) return rc;
    k_fd_up_leaf<M, kFdRegQ><<<dim3(ngroups, nchunk), f.ncol * q, smem, st>>>(s, f, dct, ppc, h0);
  } else {
    static size_t cap[64] = {};
    eo_status rc = ensure_smem((const void*)k_fd_up_leaf<M, 0>, smem, cap, 0);
    if (rc) return rc;
    k_fd_up_leaf<M, 0><<<dim3(ngroups, nchunk), f.ncol * q, smem, st>>>(s, f, dct, ppc, h0);
  }
  EO_CUDA_TRY(cudaGetLastError());
  return EO_OK;
}

template <class M>
eo_status down_leaf_t(Handle& h, const Sweep& s, const FdArgs& f, int& nchunk, cudaStream_t st) {
  const int q = f.q, qq = q * q;
  typename M::CT* wd = (typename M::CT*)h.fd_wd;
  const size_t tot = (size_t)s.P * s.K * qq;
  k_fd_wd<M><<<(unsigned)std::min<size_t>(4096, (tot + 255) / 256), 256, 0, st>>>(s.P, s.p0, s.K, qq, s.wgt,
                                                                                 h.fd_dinv, wd);
  EO_CUDA_TRY(cudaGetLastError());
  const int ng = s.K * s.K * qq;
  k_fd_gsum<<<(ng + 31) / 32, 1024, 0, st>>>(s.P, s.p0, s.K, qq, s.wgt, s.coef, h.fd_dinv, h.fd_gsum);
  EO_CUDA_TRY(cudaGetLastError());
  const int ncols = f.nleaf * s.R;
  const int ngroups = (ncols + f.ncol - 1) / f.ncol;
  nchunk = std::max(1, std::min(s.P, (608 + ngroups - 1) / ngroups));
  nchunk = std::min(nchunk, h.nchunk);
  const int ppc = (s.P + nchunk - 1) / nchunk;
  nchunk = (s.P + ppc - 1) / ppc;
  const size_t smem = fd_down_smem(q, s.K, f.ncol);
  if (fd_down_reg(q, s.K)) {
    static size_t cap[64] = {};
    eo_status rc = ensure_smem((const void*)k_fd_down_leaf<M, kFdRegQ>, smem, cap, 0);
    if (rc) return rc;
    k_fd_down_leaf<M, kFdRegQ><<<dim3(ngroups, nchunk), f.ncol * q, smem, st>>>(s, f, wd, h.lv[0].bseg, ppc, h.E,
                                                                              h.part);
  } else {
    static size_t cap[64] = {};
    eo_status rc = ensure_smem((const void*)k_fd_down_leaf<M, 0>, smem, cap, 0);
    if (rc) return rc;
    k_fd_down_leaf<M, 0><<<dim3(ngroups, nchunk), f.ncol * q, smem, st>>>(s, f, wd, h.lv[0].bseg, ppc, h.E, h.part);
  }
  EO_CUDA_TRY(cudaGetLastError());
  return EO_OK;
}

}  // namespace

eo_status fd_up_kernel(Handle& h, const Sweep& s, int nleaf, cd* h0, int ncol, cudaStream_t st) {
  FdArgs f = fd_args(h, nleaf, ncol);
  return h.fd_pair ? up_leaf_t<Pair>(h, s, f, h0, st) : up_leaf_t<F64>(h, s, f, h0, st);
}

eo_status fd_up_leaf(Handle& h, const Sweep& s, int nleaf, cd* h0, cudaStream_t st) {
  const int qq = h.g.q * h.g.q;
  FdArgs f = fd_args(h, nleaf, h.fd_ncol_up);
  k_fd_src<<<dim3(nleaf, s.R), 256, sizeof(double) * 4 * qq, st>>>(s, f, h.fd_ghat);
  EO_CUDA_TRY(cudaGetLastError());
  return fd_up_kernel(h, s, nleaf, h0, h.fd_ncol_up, st);
}

eo_status fd_down_leaf(Handle& h, const Sweep& s, int nleaf, int ncol, int& nchunk, cudaStream_t st) {
  FdArgs f = fd_args(h, nleaf, ncol);
  return h.fd_pair ? down_leaf_t<Pair>(h, s, f, nchunk, st) : down_leaf_t<F64>(h, s, f, nchunk, st);
}

// columns per block the leaf kernels can take at this q (block <= 256 threads,
// shared memory <= 200 KB)
std::vector<int> fd_ncol_candidates(const Handle& h) {
  std::vector<int> v;
  const int q = h.g.q;
  for (int nc : {2, 3, 4, 6, 9, 12, 16}) {
    if (nc * q > 256) continue;
    if (fd_up_smem(q, h.K, nc) > 200 * 1024 || fd_down_smem(q, h.K, nc) > 200 * 1024) continue;
    v.push_back(nc);
  }
  return v;
}

// Build-time setup from the leaf-0 real matrices the dense build assembled
// (device, column-major: Aii0 ni x ni, Aib ni x nb, Fbi nb x ni).  Checks that
// they are the separable forms this path assumes, then uploads the basis, the
// 1-D coupling and flux vectors in that basis, dinv for every pole and
// coef * dinv.
eo_status fd_setup(Handle& h, const double* dAii0, const double* dAib, const double* dFbi, cudaStream_t st) {
  const int p = h.g.p, q = h.g.q, qq = q * q, ni = qq, nb = 4 * q;
  std::vector<double> Aii0((size_t)ni * ni), Aib((size_t)ni * nb), Fbi((size_t)nb * ni);
  EO_CUDA_TRY(cudaMemcpyAsync(Aii0.data(), dAii0, sizeof(double) * Aii0.size(), cudaMemcpyDeviceToHost, st));
  EO_CUDA_TRY(cudaMemcpyAsync(Aib.data(), dAib, sizeof(double) * Aib.size(), cudaMemcpyDeviceToHost, st));
  EO_CUDA_TRY(cudaMemcpyAsync(Fbi.data(), dFbi, sizeof(double) * Fbi.size(), cudaMemcpyDeviceToHost, st));
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  const double* Dx = h.Dx;
  const double* Dy = h.Dy;
  std::vector<double> DDx((size_t)p * p, 0.0), DDy((size_t)p * p, 0.0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      for (int l = 0; l < p; ++l) {
        DDx[i * p + j] += Dx[i * p + l] * Dx[l * p + j];
        DDy[i * p + j] += Dy[i * p + l] * Dy[l * p + j];
      }
  std::vector<double> Mx((size_t)qq), My((size_t)qq);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      Mx[i * q + j] = DDx[(i + 1) * p + (j + 1)];
      My[i * q + j] = DDy[(i + 1) * p + (j + 1)];
    }
  // 1-D boundary coupling (interior row k or j) and flux (outward normal) vectors
  std::vector<double> cW(q), cE(q), cS(q), cN(q), rS(q), rN(q), rE(q), rW(q);
  for (int i = 0; i < q; ++i) {
    cW[i] = DDx[(i + 1) * p + 0];
    cE[i] = DDx[(i + 1) * p + (p - 1)];
    cS[i] = DDy[(i + 1) * p + 0];
    cN[i] = DDy[(i + 1) * p + (p - 1)];
    rS[i] = -Dy[0 * p + (i + 1)];
    rN[i] = Dy[(p - 1) * p + (i + 1)];
    rE[i] = Dx[(p - 1) * p + (i + 1)];
    rW[i] = -Dx[0 * p + (i + 1)];
  }
  // the assembled leaf must be exactly these separable forms
  double amax = 0.0, err = 0.0;
  for (int c = 0; c < ni; ++c)
    for (int r = 0; r < ni; ++r) {
      const int k = r % q, j = r / q, k2 = c % q, j2 = c / q;
      const double v = (j == j2 ? Mx[k * q + k2] : 0.0) + (k == k2 ? My[j * q + j2] : 0.0);
      amax = std::max(amax, std::fabs(Aii0[r + (size_t)c * ni]));
      err = std::max(err, std::fabs(Aii0[r + (size_t)c * ni] - v));
    }
  for (int bi = 0; bi < nb; ++bi)
    for (int r = 0; r < ni; ++r) {
      const int k = r % q, j = r / q, side = bi / q, o = bi % q;
      double v = 0.0;
      if (side == 0) v = (k == o) ? cS[j] : 0.0;
      else if (side == 1) v = (j == o) ? cE[k] : 0.0;
      else if (side == 2) v = (k == o) ? cN[j] : 0.0;
      else v = (j == o) ? cW[k] : 0.0;
      err = std::max(err, std::fabs(Aib[r + (size_t)bi * ni] - v));
    }
  double fmax = 0.0, ferr = 0.0;
  for (int r = 0; r < ni; ++r)
    for (int t = 0; t < nb; ++t) {
      const int k = r % q, j = r / q, side = t / q, o = t % q;
      double v = 0.0;
      if (side == 0) v = (k == o) ? rS[j] : 0.0;
      else if (side == 1) v = (j == o) ? rE[k] : 0.0;
      else if (side == 2) v = (k == o) ? rN[j] : 0.0;
      else v = (j == o) ? rW[k] : 0.0;
      fmax = std::max(fmax, std::fabs(Fbi[t + (size_t)r * nb]));
      ferr = std::max(ferr, std::fabs(Fbi[t + (size_t)r * nb] - v));
    }
  if (err > 1e-12 * amax || ferr > 1e-12 * fmax)
    return fail(EO_ERR_UNSUPPORTED, "fast-diagonal leaves: the leaf operator is not separable (" +
                                        std::to_string(err / amax) + ", " + std::to_string(ferr / fmax) + ")");
  std::vector<double> lx, Vx, Vxi, ly, Vy, Vyi;
  eo_status rc = real_eigen(q, Mx, lx, Vx, Vxi);
  if (rc) return rc;
  if ((rc = real_eigen(q, My, ly, Vy, Vyi))) return rc;
  const FdLayout Lo{q, qq};
  std::vector<double> cst(Lo.size(), 0.0);
  std::copy(Vx.begin(), Vx.end(), cst.begin() + Lo.Vx());
  std::copy(Vxi.begin(), Vxi.end(), cst.begin() + Lo.Vxi());
  std::copy(Vy.begin(), Vy.end(), cst.begin() + Lo.Vy());
  std::copy(Vyi.begin(), Vyi.end(), cst.begin() + Lo.Vyi());
  std::copy(lx.begin(), lx.end(), cst.begin() + Lo.lx());
  std::copy(ly.begin(), ly.end(), cst.begin() + Lo.ly());
  for (int a = 0; a < q; ++a) {
    double w = 0, e = 0, s = 0, n = 0, rs = 0, rn = 0, re = 0, rw = 0;
    for (int m = 0; m < q; ++m) {
      w += Vxi[a * q + m] * cW[m];
      e += Vxi[a * q + m] * cE[m];
      s += Vyi[a * q + m] * cS[m];
      n += Vyi[a * q + m] * cN[m];
      rs += rS[m] * Vy[m * q + a];
      rn += rN[m] * Vy[m * q + a];
      re += rE[m] * Vx[m * q + a];
      rw += rW[m] * Vx[m * q + a];
    }
    cst[Lo.cW() + a] = w; cst[Lo.cE() + a] = e; cst[Lo.cS() + a] = s; cst[Lo.cN() + a] = n;
    cst[Lo.rS() + a] = rs; cst[Lo.rN() + a] = rn; cst[Lo.rE() + a] = re; cst[Lo.rW() + a] = rw;
  }
  EO_CUDA_TRY(cudaMemcpyAsync(h.fd_c, cst.data(), sizeof(double) * cst.size(), cudaMemcpyHostToDevice, st));
  std::vector<cd> dinv((size_t)h.P * qq);
  for (int j = 0; j < h.P; ++j) {
    const std::complex<double> k2 = kappa2(h, j);
    for (int b = 0; b < q; ++b)
      for (int a = 0; a < q; ++a) {
        const std::complex<double> d = 1.0 / (lx[a] + ly[b] - k2);
        dinv[(size_t)j * qq + b * q + a] = make_double2(d.real(), d.imag());
      }
  }
  EO_CUDA_TRY(cudaMemcpyAsync(h.fd_dinv, dinv.data(), sizeof(cd) * dinv.size(), cudaMemcpyHostToDevice, st));
  const size_t tot = (size_t)h.P * h.K * qq;
  const unsigned nbk = (unsigned)std::min<size_t>(4096, (tot + 255) / 256);
  if (h.fd_pair) k_fd_dc<Pair><<<nbk, 256, 0, st>>>(h.P, h.K, qq, h.coef, h.fd_dinv, (float4*)h.fd_dc);
  else k_fd_dc<F64><<<nbk, 256, 0, st>>>(h.P, h.K, qq, h.coef, h.fd_dinv, h.fd_dc);
  EO_CUDA_TRY(cudaGetLastError());
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  return EO_OK;
}

}  // namespace eo
