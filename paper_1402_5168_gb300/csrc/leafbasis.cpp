// Separable eigenbasis of a constant-coefficient leaf (host side).
//
// On a leaf with a constant coefficient a, the interior block of the
// collocated operator div(a grad) (Section 2.2, nested 1-D differentiation)
// is a Kronecker sum
//     A_ii = I_y (x) M_x + M_y (x) I_x,   M_x = a (D_x D_x)_ii,  M_y = a (D_y D_y)_ii
// (interior rows and columns of the squared, scaled Chebyshev differentiation
// matrix).  With M_x = V_x diag(lx) V_x^{-1} and M_y = V_y diag(ly) V_y^{-1},
//     A_ii - kappa^2 = (V_y (x) V_x) diag(lx_a + ly_b - kappa^2) (V_y (x) V_x)^{-1},
// so every leaf solve of every pole is a change of basis, a pointwise division
// and the inverse change of basis ("fast diagonalisation").  The boundary
// coupling A_ib and the flux rows F_bi of such a leaf are sums of outer products
// of 1-D vectors, so they also act through q-vectors in that basis.
//
// The eigenvalues of the interior block of a squared Chebyshev differentiation
// matrix are real, negative and distinct; real_eigen below relies on that and
// reports EO_ERR_UNSUPPORTED otherwise.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "engine.h"

namespace eo {

namespace {

// Solve (A) x = b in place for one right-hand side by LU with partial pivoting
// (A row-major n x n, overwritten).  Tiny pivots are replaced by tiny * scale so
// that inverse iteration on a (numerically) singular shift still returns the
// dominant direction.
void lu_solve(int n, std::vector<double>& A, std::vector<double>& b, double scale) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int r = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[r * n + k])) r = i;
    piv[k] = r;
    if (r != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[r * n + j]);
      std::swap(b[k], b[r]);
    }
    if (std::fabs(A[k * n + k]) < 1e-300 + 1e-15 * scale) A[k * n + k] = 1e-15 * scale;
    for (int i = k + 1; i < n; ++i) {
      const double f = A[i * n + k] / A[k * n + k];
      A[i * n + k] = 0.0;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];
    b[k] = s / A[k * n + k];
  }
}

// Inverse of a row-major n x n matrix by Gauss-Jordan elimination with partial
// pivoting.  Returns false if a pivot vanishes.
bool invert(int n, const std::vector<double>& A0, std::vector<double>& Ainv) {
  std::vector<double> A = A0;
  Ainv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Ainv[i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int r = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[r * n + k])) r = i;
    if (A[r * n + k] == 0.0) return false;
    if (r != k)
      for (int j = 0; j < n; ++j) {
        std::swap(A[k * n + j], A[r * n + j]);
        std::swap(Ainv[k * n + j], Ainv[r * n + j]);
      }
    const double d = 1.0 / A[k * n + k];
    for (int j = 0; j < n; ++j) { A[k * n + j] *= d; Ainv[k * n + j] *= d; }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = A[i * n + k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[i * n + j] -= f * A[k * n + j];
        Ainv[i * n + j] -= f * Ainv[k * n + j];
      }
    }
  }
  return true;
}

// Eigenvalues of a real matrix with real eigenvalues: Householder reduction to
// upper Hessenberg form, then shifted QR steps (Givens rotations) with the
// eigenvalue of the trailing 2x2 block nearest its last diagonal entry as the
// shift, deflating from the bottom.  Returns false if a 2x2 block with complex
// eigenvalues remains or the iteration does not converge.
bool hessenberg_qr_eigenvalues(int n, const std::vector<double>& M, std::vector<double>& lam) {
  std::vector<double> H = M;
  auto at = [&](int i, int j) -> double& { return H[(size_t)i * n + j]; };
  // Householder reduction
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += at(i, k) * at(i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    if (at(k + 1, k) > 0) alpha = -alpha;
    std::vector<double> v(n, 0.0);
    v[k + 1] = at(k + 1, k) - alpha;
    for (int i = k + 2; i < n; ++i) v[i] = at(i, k);
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
    if (vn == 0.0) continue;
    // H = (I - 2 v v^T / vn) H (I - 2 v v^T / vn)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = k + 1; i < n; ++i) s += v[i] * at(i, j);
      s *= 2.0 / vn;
      for (int i = k + 1; i < n; ++i) at(i, j) -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += at(i, j) * v[j];
      s *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) at(i, j) -= s * v[j];
    }
    for (int i = k + 2; i < n; ++i) at(i, k) = 0.0;
  }
  lam.assign(n, 0.0);
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0, total = 0;
  std::vector<double> cs(n), sn(n);
  while (hi >= 0) {
    if (hi == 0) { lam[0] = at(0, 0); break; }
    // find the start of the unreduced block ending at hi
    int lo = hi;
    while (lo > 0) {
      const double s = std::fabs(at(lo - 1, lo - 1)) + std::fabs(at(lo, lo));
      if (std::fabs(at(lo, lo - 1)) <= eps * (s > 0 ? s : 1.0)) { at(lo, lo - 1) = 0.0; break; }
      --lo;
    }
    if (lo == hi) { lam[hi] = at(hi, hi); --hi; iter = 0; continue; }
    if (++iter > 100 || ++total > 100 * n) return false;
    // shift: eigenvalue of the trailing 2x2 block nearest at(hi, hi)
    const double a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
    const double disc = 0.25 * (a - d) * (a - d) + b * c;
    double mu = d;
    if (disc >= 0) {
      const double r = std::sqrt(disc), m = 0.5 * (a + d);
      mu = (std::fabs(m + r - d) < std::fabs(m - r - d)) ? m + r : m - r;
    }
    if (iter % 11 == 10) mu = d + 0.75 * std::fabs(c);   // exceptional shift
    // QR step on the block [lo, hi]: H - mu I = QR, H <- RQ + mu I
    for (int i = lo; i <= hi; ++i) at(i, i) -= mu;
    for (int k = lo; k < hi; ++k) {
      const double x = at(k, k), y = at(k + 1, k);
      const double r = std::hypot(x, y);
      const double cc = r == 0 ? 1.0 : x / r, ss = r == 0 ? 0.0 : y / r;
      cs[k] = cc; sn[k] = ss;
      for (int j = k; j <= hi; ++j) {
        const double t1 = at(k, j), t2 = at(k + 1, j);
        at(k, j) = cc * t1 + ss * t2;
        at(k + 1, j) = -ss * t1 + cc * t2;
      }
    }
    for (int k = lo; k < hi; ++k) {
      const double cc = cs[k], ss = sn[k];
      for (int i = lo; i <= std::min(k + 2, hi); ++i) {
        const double t1 = at(i, k), t2 = at(i, k + 1);
        at(i, k) = cc * t1 + ss * t2;
        at(i, k + 1) = -ss * t1 + cc * t2;
      }
    }
    for (int i = lo; i <= hi; ++i) at(i, i) += mu;
  }
  return true;
}

}  // namespace

// M (row-major n x n) = V diag(lam) Vinv with real lam, V's columns of unit
// 2-norm and largest-magnitude entry positive, eigenvalues in descending order.
// Verified: max|M V - V diag(lam)| and max|V Vinv - I| small, else
// EO_ERR_UNSUPPORTED.
eo_status real_eigen(int n, const std::vector<double>& M, std::vector<double>& lam, std::vector<double>& V,
                     std::vector<double>& Vinv) {
  double mmax = 0.0;
  for (double x : M) mmax = std::max(mmax, std::fabs(x));
  if (!(mmax > 0) || !std::isfinite(mmax)) return fail(EO_ERR_UNSUPPORTED, "leaf basis: zero or non-finite matrix");
  if (!hessenberg_qr_eigenvalues(n, M, lam))
    return fail(EO_ERR_UNSUPPORTED, "leaf basis: eigenvalues are not all real (QR did not deflate)");
  std::sort(lam.begin(), lam.end(), [](double x, double y) { return x > y; });
  for (int i = 0; i + 1 < n; ++i)
    if (lam[i] - lam[i + 1] <= 1e-10 * mmax)
      return fail(EO_ERR_UNSUPPORTED, "leaf basis: repeated eigenvalues");
  // eigenvectors by inverse iteration at each eigenvalue
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    std::vector<double> v(n);
    for (int k = 0; k < n; ++k) v[k] = 1.0 + 0.37 * k / n;
    for (int it = 0; it < 3; ++it) {
      std::vector<double> A = M;
      for (int k = 0; k < n; ++k) A[k * n + k] -= lam[i];
      lu_solve(n, A, v, mmax);
      double nv = 0.0;
      for (double x : v) nv += x * x;
      nv = std::sqrt(nv);
      if (!(nv > 0) || !std::isfinite(nv)) return fail(EO_ERR_UNSUPPORTED, "leaf basis: inverse iteration failed");
      for (double& x : v) x /= nv;
    }
    int km = 0;
    for (int k = 1; k < n; ++k)
      if (std::fabs(v[k]) > std::fabs(v[km])) km = k;
    const double sg = v[km] < 0 ? -1.0 : 1.0;
    for (int k = 0; k < n; ++k) V[(size_t)k * n + i] = sg * v[k];
  }
  if (!invert(n, V, Vinv)) return fail(EO_ERR_UNSUPPORTED, "leaf basis: eigenvector matrix singular");
  // refine each eigenvalue as (Vinv M V)_ii
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      double mv = 0.0;
      for (int j = 0; j < n; ++j) mv += M[(size_t)k * n + j] * V[(size_t)j * n + i];
      s += Vinv[(size_t)i * n + k] * mv;
    }
    lam[i] = s;
  }
  double r1 = 0.0, r2 = 0.0;
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < n; ++i) {
      double mv = 0.0, vv = 0.0;
      for (int j = 0; j < n; ++j) {
        mv += M[(size_t)k * n + j] * V[(size_t)j * n + i];
        vv += V[(size_t)k * n + j] * Vinv[(size_t)j * n + i];
      }
      r1 = std::max(r1, std::fabs(mv - V[(size_t)k * n + i] * lam[i]));
      r2 = std::max(r2, std::fabs(vv - (k == i ? 1.0 : 0.0)));
    }
  if (r1 > 1e-12 * mmax * n || r2 > 1e-12 * n)
    return fail(EO_ERR_UNSUPPORTED, "leaf basis: eigen-decomposition residual too large (" + std::to_string(r1 / mmax) +
                                        ", " + std::to_string(r2) + ")");
  return EO_OK;
}

// Interior block of a (D D) for a row-major p x p differentiation matrix D:
// q x q row-major, q = p - 2.
std::vector<double> interior_second_derivative(int p, const double* D, double a) {
  const int q = p - 2;
  std::vector<double> M((size_t)q * q, 0.0);
  for (int i = 1; i <= q; ++i)
    for (int j = 1; j <= q; ++j) {
      double s = 0.0;
      for (int l = 0; l < p; ++l) s += D[i * p + l] * D[l * p + j];
      M[(size_t)(i - 1) * q + (j - 1)] = a * s;
    }
  return M;
}

}  // namespace eo

extern "C" eo_status eo_leaf_basis(int p, double len, double a, double* lam, double* V, double* Vinv) {
  using namespace eo;
  if (p < 4 || p > 24) return fail(EO_ERR_INVALID_ARG, "p must be in [4, 24]");
  if (!(len > 0) || !(a > 0) || !std::isfinite(len) || !std::isfinite(a))
    return fail(EO_ERR_INVALID_ARG, "len and a must be positive and finite");
  if (!lam || !V || !Vinv) return fail(EO_ERR_INVALID_ARG, "null argument");
  Grid g;
  eo_status rc = make_grid(1, 1, p, 0.0, len, 0.0, len, g);
  if (rc) return rc;
  std::vector<double> D(g.D);
  for (double& x : D) x *= 2.0 / len;
  const int q = p - 2;
  std::vector<double> l, v, vi;
  rc = real_eigen(q, interior_second_derivative(p, D.data(), a), l, v, vi);
  if (rc) return rc;
  std::copy(l.begin(), l.end(), lam);
  std::copy(v.begin(), v.end(), V);
  std::copy(vi.begin(), vi.end(), Vinv);
  set_error("");
  return EO_OK;
}
