// Device helpers and argument structs shared by the forward sweeps (apply.cu)
// and the transposed sweeps (adjoint.cu).
#pragma once

#include <cstdint>

#include "handle.h"

namespace eo {

__device__ __forceinline__ cd cmul(cd a, cd b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cfma(cd& acc, cd a, cd b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// Operator storage type TA:
//   double2 -- FP64 blocks, FP64 products;
//   float2  -- FP32 blocks, FP32 products and sums;
//   float4  -- FP32 pairs (re_hi, im_hi, re_lo, im_lo) holding an FP64 value to
//              ~2^-48: products split exactly with fma (p = x_h y_h, e = fma(x_h,
//              y_h, -p)), hi parts summed with an error-free two-sum, the small
//              cross terms in a plain FP32 sum.  This runs on the FP32 pipe at
//              near-FP64 accuracy (GB300's FP64 pipe is ~60x slower than FP32).
// Vectors enter the products in the same type (Cv::from); Acc holds the sums
// and returns them as FP64 (Cv::to).  Part is a partial sum of one k group in the
// cross-group reduction of cmv (16 bytes, the size of a cd): FP64 for double2 and
// float2; for float4 the renormalised FP32 pair, so that the reduction stays on the
// FP32 pipe and only the final sum is converted to FP64.
template <typename TA> struct Cv;
template <> struct Cv<double2> {
  typedef double2 Acc;
  typedef cd Part;
  __device__ static double2 from(cd v) { return v; }
  __device__ static cd to(const Acc& v) { return v; }
  __device__ static Part part(const Acc& v) { return v; }
  __device__ static void part_add(Part& s, const Part& v) { s.x += v.x; s.y += v.y; }
  __device__ static cd part_to(const Part& v) { return v; }
  __device__ static Acc zero() { return make_double2(0.0, 0.0); }
  __device__ static void mac(Acc& acc, const double2& a, const double2& b) { cfma(acc, a, b); }
};
template <> struct Cv<float2> {
  typedef float2 Acc;
  typedef cd Part;
  __device__ static float2 from(cd v) { return make_float2((float)v.x, (float)v.y); }
  __device__ static cd to(const Acc& v) { return make_double2(v.x, v.y); }
  __device__ static Part part(const Acc& v) { return to(v); }
  __device__ static void part_add(Part& s, const Part& v) { s.x += v.x; s.y += v.y; }
  __device__ static cd part_to(const Part& v) { return v; }
  __device__ static Acc zero() { return make_float2(0.f, 0.f); }
  __device__ static void mac(Acc& acc, const float2& a, const float2& b) { cfma(acc, a, b); }
};

struct DFAcc {
  float sr, cr, lr, si, ci, li;   // hi sum, two-sum compensation, cross-term sum (re, im)
};
__device__ __forceinline__ void df_two_sum(float& s, float& c, float p) {
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
  s = t;
}
// x*y for x = xh + xl, y = yh + yl: p + lo with p = fl(xh yh) and lo the rest to ~2^-48
__device__ __forceinline__ void df_prod(float xh, float xl, float yh, float yl, float& p, float& lo) {
  p = __fmul_rn(xh, yh);
  const float e = __fmaf_rn(xh, yh, -p);
  lo = __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, e));
}
// (hi, lo) = a + b exactly (two-sum, no ordering assumption)
__device__ __forceinline__ void df_renorm(float a, float b, float& hi, float& lo) {
  hi = __fadd_rn(a, b);
  const float bp = __fsub_rn(hi, a);
  lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bp)), __fsub_rn(b, bp));
}
// s = s + v for FP32 pairs (hi, lo): the error of the hi sum and both lo parts join a
// renormalised lo (about 2^-47 of the larger operand)
__device__ __forceinline__ void df_pair_add(float& sh, float& sl, float vh, float vl) {
  float c = 0.f;
  df_two_sum(sh, c, vh);
  df_renorm(sh, __fadd_rn(c, __fadd_rn(sl, vl)), sh, sl);
}
template <> struct Cv<float4> {
  typedef DFAcc Acc;
  typedef float4 Part;   // (re_hi, im_hi, re_lo, im_lo)
  __device__ static float4 from(cd v) {
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    return make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
  }
  __device__ static cd to(const Acc& a) {
    return make_double2((double)a.sr + ((double)a.cr + (double)a.lr), (double)a.si + ((double)a.ci + (double)a.li));
  }
  __device__ static Acc zero() { return DFAcc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f}; }
  __device__ static Part part(const Acc& a) {
    float rh, rl, ih, il;
    df_renorm(a.sr, __fadd_rn(a.cr, a.lr), rh, rl);
    df_renorm(a.si, __fadd_rn(a.ci, a.li), ih, il);
    return make_float4(rh, ih, rl, il);
  }
  __device__ static void part_add(Part& s, const Part& v) {
    df_pair_add(s.x, s.z, v.x, v.z);
    df_pair_add(s.y, s.w, v.y, v.w);
  }
  __device__ static cd part_to(const Part& v) {
    return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  }
  // re += a_re b_re - a_im b_im ; im += a_re b_im + a_im b_re
  __device__ static void mac(Acc& acc, const float4& a, const float4& b) {
    float p, lo;
    df_prod(a.x, a.z, b.x, b.z, p, lo);
    df_two_sum(acc.sr, acc.cr, p);
    acc.lr = __fadd_rn(acc.lr, lo);
    df_prod(a.y, a.w, b.y, b.w, p, lo);
    df_two_sum(acc.sr, acc.cr, -p);
    acc.lr = __fsub_rn(acc.lr, lo);
    df_prod(a.x, a.z, b.y, b.w, p, lo);
    df_two_sum(acc.si, acc.ci, p);
    acc.li = __fadd_rn(acc.li, lo);
    df_prod(a.y, a.w, b.x, b.z, p, lo);
    df_two_sum(acc.si, acc.ci, p);
    acc.li = __fadd_rn(acc.li, lo);
  }
};
__device__ __forceinline__ float2 operator_ld(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 operator_ld(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float4 operator_ld(const float4* p) { return __ldg(p); }

// 16-byte aligned pointer past n elements of T
template <typename T>
__device__ __forceinline__ cd* after(T* base, size_t n) {
  return (cd*)(((uintptr_t)(base + n) + 15) & ~(uintptr_t)15);
}

// Rows per pass of cmv: the rows split into the fewest passes of at most 256,
// each rounded up to a multiple of 16 (half-warps stay on one k group).
__host__ __device__ __forceinline__ int cmv_rp(int rows) {
  const int npass = (rows + 255) / 256;
  return (((rows + npass - 1) / npass) + 15) & ~15;
}
// Threads of a block that runs cmv over `rows`: rp rows times the k groups that fit in 256.
inline int cmv_threads(int rows) {
  const int rp = cmv_rp(rows);
  return rp * (256 / rp);
}

// Complex FP32 pairs (re_hi, im_hi, re_lo, im_lo), the layout of Cv<float4>: sums on the
// FP32 pipe (the FP64 pipe of GB300 runs at about 1/64 of its rate).
__device__ __forceinline__ float4 cp_add(float4 a, const float4& b) {
  df_pair_add(a.x, a.z, b.x, b.z);
  df_pair_add(a.y, a.w, b.y, b.w);
  return a;
}
__device__ __forceinline__ float4 cp_scale(const float4& a, float s) {   // s a power of two (exact)
  return make_float4(s * a.x, s * a.y, s * a.z, s * a.w);
}
__device__ __forceinline__ cd cp_to(const float4& a) {
  return make_double2((double)a.x + (double)a.z, (double)a.y + (double)a.w);
}

// C[c][r] = sum_{j<k} A[r + j*lda] B[c][j]  for r < rows, c < NC.
// Bs: shared [NC][kb]; Cs: shared [NC][rows]; red: shared [256 * NC].
// blockDim.x >= cmv_rp(rows); threads beyond rp * (blockDim.x / rp) idle.
// RAW: Cs receives Cv<TA>::Part values (for FP32 pairs the pair itself, no FP64
// conversion) in the slots of the cd entries.
template <int NC, typename TA, bool RAW = false>
__device__ void cmv(const TA* __restrict__ A, int lda, int rows, int k, const TA* Bs, int kb,
                    cd* Cs, cd* red) {
  const int nt = blockDim.x, t = threadIdx.x;
  const int rp = cmv_rp(rows);
  const int ks = nt / rp;
  const int ri = t % rp, kg = t / rp;
  for (int r0 = 0; r0 < rows; r0 += rp) {
    const int r = r0 + ri;
    typename Cv<TA>::Acc acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = Cv<TA>::zero();
    if (kg < ks && r < rows) {
      const TA* Ar = A + r;
      int j = kg;
      for (; j + 3 * ks < k; j += 4 * ks) {
        const TA a0 = operator_ld(Ar + (size_t)j * lda);
        const TA a1 = operator_ld(Ar + (size_t)(j + ks) * lda);
        const TA a2 = operator_ld(Ar + (size_t)(j + 2 * ks) * lda);
        const TA a3 = operator_ld(Ar + (size_t)(j + 3 * ks) * lda);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          Cv<TA>::mac(acc[c], a0, Bs[c * kb + j]);
          Cv<TA>::mac(acc[c], a1, Bs[c * kb + j + ks]);
          Cv<TA>::mac(acc[c], a2, Bs[c * kb + j + 2 * ks]);
          Cv<TA>::mac(acc[c], a3, Bs[c * kb + j + 3 * ks]);
        }
      }
      for (; j < k; j += ks) {
        const TA a = operator_ld(Ar + (size_t)j * lda);
#pragma unroll
        for (int c = 0; c < NC; ++c) Cv<TA>::mac(acc[c], a, Bs[c * kb + j]);
      }
    }
    typedef typename Cv<TA>::Part Part;
    static_assert(sizeof(Part) == sizeof(cd), "a partial sum takes the slot of a cd");
    if (ks == 1) {
      if (r < rows)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (RAW) reinterpret_cast<Part*>(Cs)[c * rows + r] = Cv<TA>::part(acc[c]);
          else Cs[c * rows + r] = Cv<TA>::to(acc[c]);
        }
    } else {
      Part* pr = reinterpret_cast<Part*>(red);
      if (kg < ks)
#pragma unroll
        for (int c = 0; c < NC; ++c) pr[(kg * NC + c) * rp + ri] = Cv<TA>::part(acc[c]);
      __syncthreads();
      if (kg == 0 && r < rows) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          Part s = pr[c * rp + ri];
          for (int g = 1; g < ks; ++g) Cv<TA>::part_add(s, pr[(g * NC + c) * rp + ri]);
          if (RAW) reinterpret_cast<Part*>(Cs)[c * rows + r] = s;
          else Cs[c * rows + r] = Cv<TA>::part_to(s);
        }
      }
    }
    __syncthreads();
  }
}

// Kernel arguments shared by the sweep kernels.
struct Sweep {
  int R;                 // right-hand sides in this call
  int P;                 // poles in this call (local index pl, operator index p0 + pl)
  int p0;
  int q, ni, nb;
  long long n_int, n_edge, n_nodes;
  int shared;
  // pre-map sources (real, per rhs stride), K of them, and coefficients [P][K]
  int K;
  const double* src[3];
  long long src_rs[3];
  const cd* coef;
  const cd* wgt;
};

__device__ __forceinline__ void col_box(int c, int R, int& box, int& r) {
  box = c / R;
  r = c - box * R;
}

struct MergeArgs {
  int nbox, nbx, nbx_c, nbox_c, dir, nbd, nbd_c, n3, zu_rows;
  const int* par_child;
  const int* par_idx;
  const int* a3;
  const int* b3;
  const void* ZU;
  long long zps, zbs;
  const void* S;
  long long sps, sbs;
  const int* bseg;
  const int* iseg;
  int nseg;
  cd* w3;
  // reflection-symmetric level (constant coefficient, shared operators): the box
  // is symmetric under Ra (across the interface line; swaps the children, fixes
  // the interface) and Rb (along it; reverses the interface, t -> n3 - 1 - t).
  // ZUs: [P][2][rh x n3h] (even, odd; rows n3h of -Z then nbq of U), Ss:
  // [P][2][n3h x nbq]; orbit maps of the parent boundary under {1, Ra, Rb, RaRb}:
  // orb[i] (orbit), osg[i] (+1 for i = rep or Ra rep, -1 for Rb rep, Ra Rb rep),
  // mem[4 r + g] (members).
  int sym = 0, n3h = 0, nbq = 0, rh = 0;
  const void* ZUs = nullptr;
  long long zsps = 0;
  const void* Ss = nullptr;
  long long ssps = 0;
  const int* orb = nullptr;
  const int* osg = nullptr;
  const int* mem = nullptr;
};

__device__ __forceinline__ void children(const MergeArgs& m, int box, int& ca, int& cb) {
  const int bx = box % m.nbx, by = box / m.nbx;
  if (m.dir == 0) { ca = by * m.nbx_c + 2 * bx; cb = ca + 1; }
  else { ca = (2 * by) * m.nbx_c + bx; cb = ca + m.nbx_c; }
}

struct RootArgs {
  int n, q, sxq, syq;
  const int* bseg;
  const void* Binv;
  const cd* bcoef;   // [P][4][2]
  const cd* nu;      // [P][4]
  const double* state;
  int F;
  // rotation-symmetric root (square walled domain): nq = n / 4 nodes per side, Binv
  // holds the four Fourier blocks [P][4][nq x nq]; c4idx[k * nq + s] is the wall
  // index of node s of side k in counterclockwise order, c4inv its inverse.  nq = 0:
  // Binv is the dense [P][n x n] inverse.
  int nq = 0;
  const int* c4idx = nullptr;
  const int* c4inv = nullptr;
};

// sign of the wall rows of side k (S, E, N, W) relative to the rotation-covariant
// form alpha d_n h + tau f d_t h (outward normal, counterclockwise tangent)
__host__ __device__ __forceinline__ double c4_sign(int k) { return (k == 1 || k == 2) ? 1.0 : -1.0; }

// v * i^j (j = 0..3)
__device__ __forceinline__ cd times_ipow(cd v, int j) {
  switch (j & 3) {
    case 0: return v;
    case 1: return make_double2(-v.y, v.x);
    case 2: return make_double2(-v.x, -v.y);
    default: return make_double2(v.y, -v.x);
  }
}

struct LeafGeo {
  int nlx, nly, p, q;
  long long n_int, n_hseg;
  const double* Dx;   // p x p row-major (scaled)
  const double* Dy;
  const double* Ex;   // q x q
  const double* Ey;
  int per = 0;        // periodic square: the top / right edge lines are lines 0
};

// global node id of local node (k, j) of leaf (a, b) in the public numbering; -1 at a corner
__device__ __forceinline__ long long gnode(const LeafGeo& g, int a, int b, int k, int j) {
  const int p = g.p, q = g.q;
  const bool kin = k > 0 && k < p - 1, jin = j > 0 && j < p - 1;
  if (kin && jin) return ((long long)b * g.nlx + a) * q * q + (long long)(j - 1) * q + (k - 1);
  if (kin) {
    const int e = j == 0 ? b : ((g.per && b + 1 == g.nly) ? 0 : b + 1);
    return g.n_int + ((long long)e * g.nlx + a) * q + (k - 1);
  }
  if (jin) {
    const int nvl = g.per ? g.nlx : g.nlx + 1;
    const int e = k == 0 ? a : ((g.per && a + 1 == g.nlx) ? 0 : a + 1);
    return g.n_int + (g.n_hseg + (long long)b * nvl + e) * q + (j - 1);
  }
  return -1;
}

// derivatives of a leaf-local field f[j*p+k] (corners unused)
__device__ __forceinline__ double ddx(const LeafGeo& g, const double* f, int k, int j) {
  double s = 0;
  for (int m = 0; m < g.p; ++m) s += g.Dx[k * g.p + m] * f[j * g.p + m];
  return s;
}
__device__ __forceinline__ double ddy(const LeafGeo& g, const double* f, int k, int j) {
  double s = 0;
  for (int m = 0; m < g.p; ++m) s += g.Dy[j * g.p + m] * f[m * g.p + k];
  return s;
}

}  // namespace eo
