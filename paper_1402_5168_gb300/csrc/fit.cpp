// Rational approximant of e^{i x} on [-X, X] (Section 1.2, eqs. def_RM,
// RM_prop1, RM_prop2).
//
// Poles on one conjugate-closed vertical line in the right half-plane,
// alpha_m = sigma + i s m (m = -M..M).  With b_{-m} = conj(b_m) the function
// R(i x) = sum_m b_m / (i x - alpha_m) satisfies R(-i x) = conj(R(i x)), so the
// residues are fitted on [0, X] by real linear least squares (Householder QR)
// in the real unknowns (b_0, Re b_1, Im b_1, ...), minimum-norm solution by
// truncated SVD.  A candidate (sigma, s, X)
// is accepted when max |e^{ix} - R(ix)| <= delta/2 on [0, X], every |b_m| <= 100
// (large residues cancel in the pole sum and amplify rounding), and
// max |R(iy)| <= 1 + delta/10 on a grid of [0, Y] with Y far beyond the poles;
// b is then divided by max(1, max|R|) so eq. RM_prop2 holds on that grid.
// The search keeps the widest X for the requested pole count.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <functional>
#include <thread>

#include "engine.h"

namespace eo {

using cplx = std::complex<double>;

// Least squares min |A x - t| for column-major A (m x n), m >= n, by Householder
// QR.  A and t are overwritten.  Returns false on a zero column.
static bool lsq(std::vector<double>& A, std::vector<double>& t, int m, int n,
                std::vector<double>& x) {
  for (int k = 0; k < n; ++k) {
    double* a = &A[(size_t)k * m];
    double nrm = 0;
    for (int i = k; i < m; ++i) nrm += a[i] * a[i];
    nrm = std::sqrt(nrm);
    if (nrm == 0) return false;
    const double alpha = a[k] > 0 ? -nrm : nrm;
    // v = a[k:] - alpha e_k, stored in a[k:]
    a[k] -= alpha;
    double vnorm2 = 0;
    for (int i = k; i < m; ++i) vnorm2 += a[i] * a[i];
    for (int j = k + 1; j < n; ++j) {
      double* c = &A[(size_t)j * m];
      double d = 0;
      for (int i = k; i < m; ++i) d += a[i] * c[i];
      const double f = 2 * d / vnorm2;
      for (int i = k; i < m; ++i) c[i] -= f * a[i];
    }
    {
      double d = 0;
      for (int i = k; i < m; ++i) d += a[i] * t[i];
      const double f = 2 * d / vnorm2;
      for (int i = k; i < m; ++i) t[i] -= f * a[i];
    }
    a[k] = alpha;   // R diagonal; the rest of v is no longer needed
    for (int i = k + 1; i < m; ++i) a[i] = 0;
  }
  // R (n x n, upper) and the first n entries of Q^T t.  The band-only problem is
  // close to rank deficient, so solve with the truncated SVD of R (singular
  // values below eps * max(m, n) * sigma_max dropped: the minimum-norm solution),
  // by one-sided Jacobi rotations on the columns of R.
  std::vector<double> U((size_t)n * n), V((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) U[(size_t)j * n + i] = (i <= j) ? A[(size_t)j * m + i] : 0.0;
    V[(size_t)j * n + j] = 1.0;
  }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double* up = &U[(size_t)p * n];
        double* uq = &U[(size_t)q * n];
        double a = 0, b = 0, c = 0;
        for (int i = 0; i < n; ++i) { a += up[i] * up[i]; b += uq[i] * uq[i]; c += up[i] * uq[i]; }
        if (c == 0 || std::abs(c) <= 1e-15 * std::sqrt(a * b)) continue;
        off = std::max(off, std::abs(c) / std::sqrt(a * b));
        const double zeta = (b - a) / (2 * c);
        const double tt = (zeta >= 0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(1 + zeta * zeta));
        const double cs = 1 / std::sqrt(1 + tt * tt), sn = cs * tt;
        for (int i = 0; i < n; ++i) {
          const double x1 = up[i], x2 = uq[i];
          up[i] = cs * x1 - sn * x2;
          uq[i] = sn * x1 + cs * x2;
        }
        double* vp = &V[(size_t)p * n];
        double* vq = &V[(size_t)q * n];
        for (int i = 0; i < n; ++i) {
          const double x1 = vp[i], x2 = vq[i];
          vp[i] = cs * x1 - sn * x2;
          vq[i] = sn * x1 + cs * x2;
        }
      }
    if (off < 1e-15) break;
  }
  // columns of U are sigma_j u_j; x = sum_j v_j (u_j . t) / sigma_j over kept j
  std::vector<double> sig(n);
  double smax = 0;
  for (int j = 0; j < n; ++j) {
    double s2 = 0;
    for (int i = 0; i < n; ++i) s2 += U[(size_t)j * n + i] * U[(size_t)j * n + i];
    sig[j] = std::sqrt(s2);
    smax = std::max(smax, sig[j]);
  }
  const double cut = 2.220446049250313e-16 * std::max(m, n) * smax;
  x.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    if (sig[j] <= cut) continue;
    double d = 0;
    for (int i = 0; i < n; ++i) d += U[(size_t)j * n + i] * t[i];
    const double f = d / (sig[j] * sig[j]);
    for (int i = 0; i < n; ++i) x[i] += f * V[(size_t)j * n + i];
  }
  return true;
}

static cplx Reval(double y, const std::vector<cplx>& al, const std::vector<cplx>& b) {
  cplx z(0.0, y), s(0.0, 0.0);
  for (size_t i = 0; i < al.size(); ++i) s += b[i] / (z - al[i]);
  return s;
}

// Residues for the pole line on [0, X]; returns false if the LS failed.
static bool residues(int N, double sigma, double s, double X, std::vector<cplx>& al,
                     std::vector<cplx>& b) {
  const int M = (N - 1) / 2;
  al.resize(N);
  for (int m = -M; m <= M; ++m) al[m + M] = cplx(sigma, s * m);
  const int ns = (int)std::ceil(X * 20.0) + 41;
  const int rows = 2 * ns, cols = N;
  std::vector<double> A((size_t)rows * cols), t(rows), x;
  for (int i = 0; i < ns; ++i) {
    const double th = X * i / (ns - 1);
    const cplx z(0.0, th);
    auto put = [&](int col, cplx v) {
      A[(size_t)col * rows + i] = v.real();
      A[(size_t)col * rows + ns + i] = v.imag();
    };
    put(0, 1.0 / (z - al[M]));
    for (int k = 1; k <= M; ++k) {
      const cplx p = 1.0 / (z - al[M + k]), n = 1.0 / (z - al[M - k]);
      put(2 * k - 1, p + n);
      put(2 * k, cplx(0, 1) * (p - n));
    }
    t[i] = std::cos(th);
    t[ns + i] = std::sin(th);
  }
  // column scaling
  std::vector<double> sc(cols);
  for (int j = 0; j < cols; ++j) {
    double s2 = 0;
    for (int i = 0; i < rows; ++i) s2 += A[(size_t)j * rows + i] * A[(size_t)j * rows + i];
    sc[j] = std::sqrt(s2);
    if (sc[j] == 0) return false;
    for (int i = 0; i < rows; ++i) A[(size_t)j * rows + i] /= sc[j];
  }
  if (!lsq(A, t, rows, cols, x)) return false;
  for (int j = 0; j < cols; ++j) x[j] /= sc[j];
  b.assign(N, cplx(0, 0));
  b[M] = x[0];
  for (int k = 1; k <= M; ++k) {
    b[M + k] = cplx(x[2 * k - 1], x[2 * k]);
    b[M - k] = std::conj(b[M + k]);
  }
  return true;
}

// Acceptance test; on success returns max |R(iy)| on the stability grid.
static bool accept(double X, double delta, const std::vector<cplx>& al,
                   const std::vector<cplx>& b, double* rmax) {
  double bmax = 0, bsum = 0, amax = 0;
  for (size_t i = 0; i < b.size(); ++i) {
    bmax = std::max(bmax, std::abs(b[i]));
    bsum += std::abs(b[i]);
    amax = std::max(amax, std::abs(al[i]));
  }
  if (bmax > 100.0) return false;
  const int nb = 1501;
  for (int i = 0; i < nb; ++i) {
    const double th = X * i / (nb - 1);
    if (std::abs(std::exp(cplx(0, th)) - Reval(th, al, b)) > 0.5 * delta) return false;
  }
  // |R(iy)| on [0, Y], spacing 0.02; beyond Y, |R| <= bsum / (y - amax) <= 1
  const double Y = std::max({50.0 * X + 200.0, 4.0 * amax + 200.0, amax + 2.0 * bsum});
  const int ny = (int)(Y / 0.02) + 1;
  double r = 0;
  for (int i = 0; i < ny; ++i) {
    r = std::max(r, std::abs(Reval(Y * i / (ny - 1), al, b)));
    if (r > 1.0 + 0.1 * delta) return false;
  }
  *rmax = r;
  return true;
}

static void store(const std::vector<cplx>& al, const std::vector<cplx>& b, double r,
                  double X, double sigma, double s, Fit& out, int E = 0) {
  out.E = E;
  const int N = (int)al.size();
  out.are.resize(N); out.aim.resize(N); out.bre.resize(N); out.bim.resize(N);
  const double scale = 1.0 / std::max(1.0, r);
  for (int i = 0; i < N; ++i) {
    out.are[i] = al[i].real(); out.aim[i] = al[i].imag();
    out.bre[i] = b[i].real() * scale; out.bim[i] = b[i].imag() * scale;
  }
  out.X = X; out.sigma = sigma; out.s = s;
}

static eo_status fit_wide_poles(int N, double delta, Fit& out);

static const double kS[] = {0.8, 0.9, 1.0, 1.1, 1.2, 1.3, 1.4, 1.5, 1.6};
static const double kRatio[] = {3.75, 4.0, 4.5, 5.0};

// Finer candidate grids, tried when the default grids give no admissible fit.
static const double kSFine[] = {0.7, 0.75, 0.8, 0.85, 0.9, 0.95, 1.0, 1.05, 1.1, 1.15, 1.2, 1.25, 1.3,
                                1.35, 1.4, 1.45, 1.5, 1.55, 1.6, 1.7, 1.8};
static const double kRatioFine[] = {3.5, 3.75, 4.0, 4.25, 4.5, 4.75, 5.0, 5.5};

static eo_status fit_for_poles_grid(int N, double delta, Fit& out, const double* ss, int ns_, const double* rs,
                                    int nr);

eo_status fit_for_poles(int N, double delta, Fit& out) {
  if (N < 3 || N % 2 == 0) return fail(EO_ERR_INVALID_ARG, "n_poles must be odd and >= 3");
  // beyond ~100 poles the dense search is slow and the wide construction is as good
  if (N > 101) {
    if (fit_wide_poles(N, delta, out) == EO_OK) return EO_OK;
  } else {
    if (fit_for_poles_grid(N, delta, out, kS, (int)(sizeof(kS) / sizeof(kS[0])), kRatio,
                           (int)(sizeof(kRatio) / sizeof(kRatio[0]))) == EO_OK)
      return EO_OK;
    if (fit_for_poles_grid(N, delta, out, kSFine, (int)(sizeof(kSFine) / sizeof(kSFine[0])), kRatioFine,
                           (int)(sizeof(kRatioFine) / sizeof(kRatioFine[0]))) == EO_OK)
      return EO_OK;
    if (fit_wide_poles(N, delta, out) == EO_OK) return EO_OK;
  }
  // Last resort: the approximant with N - 2 poles plus one more conjugate pole
  // pair on the same line with zero residues.  R is unchanged, so eqs. RM_prop1
  // and RM_prop2 hold with the band of the smaller fit.
  if (N <= 3) return fail(EO_ERR_FIT, "no admissible rational approximant for this pole count");
  Fit f;
  if (fit_for_poles(N - 2, delta, f) != EO_OK) return fail(EO_ERR_FIT, "no admissible rational approximant for this pole count");
  const int Mo = (N - 3) / 2;
  out = f;
  out.E = 0;
  out.are.insert(out.are.begin(), f.sigma);
  out.aim.insert(out.aim.begin(), -f.s * (Mo + 1));
  out.are.push_back(f.sigma);
  out.aim.push_back(f.s * (Mo + 1));
  out.bre.insert(out.bre.begin(), 0.0);
  out.bim.insert(out.bim.begin(), 0.0);
  out.bre.push_back(0.0);
  out.bim.push_back(0.0);
  set_error("");
  return EO_OK;
}

static void par_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn);

// Widest accepted band over the candidate line spacings ss and sigma/s ratios rs
// (candidates searched in parallel host threads, then the widest kept; ties go to
// the first candidate in grid order, so the result does not depend on threads).
static eo_status fit_for_poles_grid(int N, double delta, Fit& out, const double* ss, int ns_, const double* rs,
                                    int nr) {
  const int M = (N - 1) / 2;
  const int nc = ns_ * nr;
  std::vector<double> foundX(nc, 0.0);
  auto search = [&](int ci) {
    const double s = ss[ci / nr], sigma = rs[ci % nr] * s;
    std::vector<cplx> al, b;
    double X = s * M, found = 0, r = 0;
    for (; X > 0.5; X -= std::max(0.5, 0.05 * X))
      if (residues(N, sigma, s, X, al, b) && accept(X, delta, al, b, &r)) { found = X; break; }
    if (found == 0) return;
    double step = std::max(0.5, 0.05 * found) / 2;
    for (int it = 0; it < 4; ++it, step /= 2) {
      const double Xt = found + step;
      double rt;
      if (residues(N, sigma, s, Xt, al, b) && accept(Xt, delta, al, b, &rt)) found = Xt;
    }
    foundX[ci] = found;
  };
  {
    std::vector<std::thread> th;
    std::atomic<int> next(0);
    const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    for (unsigned t = 0; t < nt; ++t)
      th.emplace_back([&] {
        for (int ci = next++; ci < nc; ci = next++) search(ci);
      });
    for (auto& x : th) x.join();
  }
  int best = -1;
  for (int ci = 0; ci < nc; ++ci)
    if (foundX[ci] > 0 && (best < 0 || foundX[ci] > foundX[best])) best = ci;
  if (best < 0) return EO_ERR_FIT;
  {
    const double s = ss[best / nr], sigma = rs[best % nr] * s, X = foundX[best];
    std::vector<cplx> al, b;
    double r = 0;
    residues(N, sigma, s, X, al, b);
    accept(X, delta, al, b, &r);
    store(al, b, r, X, sigma, s, out);
  }
  return EO_OK;
}


// ---------------------------------------------------------------- wide bands
// For a band X far wider than the pole spacing the dense search above is too
// costly.  The pole line is then extended to cover [-(X + extra), X + extra] and
// the residues of all but the E outermost poles on each side are set to the
// infinite-line values b_m = beta e^{i s m}, beta = -s e^{sigma} / (2 pi): by
// Poisson summation sum_m beta e^{ism} / (i(x - s m) - sigma) = e^{ix} up to
// aliasing terms of size e^{-2 pi sigma / s} (sigma/s >= 4.5 gives < 1e-12).
// The 2E outermost residues absorb the truncation of that sum: they are the
// least-squares solution of R(ix) = e^{ix} on [0, X] with the inner residues
// held fixed.  Candidates (s, sigma/s, E, extra) are tried in a fixed order and
// accepted on the same criteria as above, with |R(iy)| checked on a grid up to
// twice the pole span and geometrically spaced points beyond.

static void par_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn) {
  unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < 4096) nt = 1;
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int64_t a = t * chunk, e = std::min<int64_t>(n, a + chunk);
    if (a >= e) break;
    th.emplace_back(fn, a, e);
  }
  for (auto& x : th) x.join();
}

static bool wide_candidate(double X, double delta, double s, double ratio, int E, double extra,
                           std::vector<cplx>& al, std::vector<cplx>& b, double* rmax) {
  const double sigma = ratio * s;
  const int M = (int)std::ceil((X + extra) / s);
  const int N = 2 * M + 1;
  if (E >= M) return false;
  al.resize(N);
  b.resize(N);
  const double beta = -s * std::exp(sigma) / (2 * M_PI);
  for (int m = -M; m <= M; ++m) {
    al[m + M] = cplx(sigma, s * m);
    b[m + M] = beta * std::exp(cplx(0.0, s * m));
  }
  // least squares for the 2E outer residues (E complex unknowns by symmetry)
  const int ns = (int)std::ceil(X * 8.0) + 41;
  const int rows = 2 * ns, cols = 2 * E;
  std::vector<double> A((size_t)rows * cols), t(rows), x;
  par_for(ns, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      const double th = X * i / (ns - 1);
      const cplx z(0.0, th);
      cplx rc(0, 0);
      for (int m = -(M - E); m <= M - E; ++m) rc += b[m + M] / (z - al[m + M]);
      const cplx tg = std::exp(cplx(0.0, th)) - rc;
      t[i] = tg.real();
      t[ns + i] = tg.imag();
      for (int k = 0; k < E; ++k) {
        const int mm = M - E + 1 + k;
        const cplx pp = 1.0 / (z - al[mm + M]), nn = 1.0 / (z - al[-mm + M]);
        const cplx c1 = pp + nn, c2 = cplx(0, 1) * (pp - nn);
        A[(size_t)(2 * k) * rows + i] = c1.real();
        A[(size_t)(2 * k) * rows + ns + i] = c1.imag();
        A[(size_t)(2 * k + 1) * rows + i] = c2.real();
        A[(size_t)(2 * k + 1) * rows + ns + i] = c2.imag();
      }
    }
  });
  std::vector<double> sc(cols);
  for (int j = 0; j < cols; ++j) {
    double s2 = 0;
    for (int i = 0; i < rows; ++i) s2 += A[(size_t)j * rows + i] * A[(size_t)j * rows + i];
    sc[j] = std::sqrt(s2);
    for (int i = 0; i < rows; ++i) A[(size_t)j * rows + i] /= sc[j];
  }
  if (!lsq(A, t, rows, cols, x)) return false;
  for (int k = 0; k < E; ++k) {
    const int mm = M - E + 1 + k;
    b[mm + M] = cplx(x[2 * k] / sc[2 * k], x[2 * k + 1] / sc[2 * k + 1]);
    b[-mm + M] = std::conj(b[mm + M]);
  }
  double bmax = 0;
  for (const cplx& v : b) bmax = std::max(bmax, std::abs(v));
  if (bmax > 100.0) return false;
  // band error and modulus on grids, in parallel
  auto maxabs = [&](int64_t n, const std::function<double(int64_t)>& f) {
    std::vector<double> part(64, 0.0);
    std::atomic<int> slot(0);
    par_for(n, [&](int64_t i0, int64_t i1) {
      double mx = 0;
      for (int64_t i = i0; i < i1; ++i) mx = std::max(mx, f(i));
      part[slot++] = mx;
    });
    return *std::max_element(part.begin(), part.end());
  };
  const int64_t nb = (int64_t)std::ceil(X / 0.02) + 1;
  const double err = maxabs(nb, [&](int64_t i) {
    const double th = X * i / (nb - 1);
    return std::abs(std::exp(cplx(0, th)) - Reval(th, al, b));
  });
  if (err > 0.5 * delta) return false;
  // |R| inside the band exceeds 1 by at most the band error; it sets the final
  // scaling too (after which the band error is at most delta)
  const double rin = maxabs(nb, [&](int64_t i) { return std::abs(Reval(X * i / (nb - 1), al, b)); });
  const double span = s * M;
  const double Y1 = 2 * span + 300.0;
  const int64_t n1 = (int64_t)std::ceil((Y1 - X) / 0.02) + 1;
  double r = maxabs(n1, [&](int64_t i) { return std::abs(Reval(X + (Y1 - X) * i / (n1 - 1), al, b)); });
  // geometric points from Y1 to 1e7, then the bound |R(iy)| <= sum|b| / (y - max|alpha|)
  const int64_t n2 = (int64_t)std::ceil(std::log(1e7 / Y1) / std::log(1.002)) + 1;
  r = std::max(r, maxabs(n2, [&](int64_t i) { return std::abs(Reval(Y1 * std::pow(1.002, (double)i), al, b)); }));
  double bsum = 0;
  for (const cplx& v : b) bsum += std::abs(v);
  if (bsum / (1e7 - std::abs(al[0])) > 1.0) return false;
  if (r > 1.0 + 0.1 * delta) return false;
  *rmax = std::max(r, rin);
  return true;
}

eo_status fit_wide(double X, double delta, Fit& out) {
  static const double cand[][4] = {
      {1.0, 4.5, 28, 32}, {1.0, 5.0, 24, 28}, {1.0, 5.0, 28, 32}, {1.2, 4.5, 16, 24}, {1.2, 4.5, 20, 28},
      {1.0, 4.5, 24, 32}, {1.0, 5.0, 20, 28}, {1.0, 4.5, 20, 28}, {1.2, 5.0, 24, 28}, {1.2, 4.5, 24, 32},
      {1.0, 5.0, 16, 24}, {1.0, 4.5, 32, 36}, {1.0, 5.0, 32, 36}, {0.8, 5.0, 32, 32}, {0.8, 4.5, 32, 32}};
  std::vector<cplx> al, b;
  for (const auto& c : cand) {
    double r = 0;
    if (wide_candidate(X, delta, c[0], c[1], (int)c[2], c[3], al, b, &r)) {
      store(al, b, r, X, c[1] * c[0], c[0], out, (int)c[2]);
      return EO_OK;
    }
  }
  return fail(EO_ERR_FIT, "no admissible wide-band rational approximant");
}

// Pole count given and beyond the dense search: the wide construction with the
// band that count covers, X = s M - extra, for the first candidate accepted.
static eo_status fit_wide_poles(int N, double delta, Fit& out) {
  static const double cand[][4] = {{1.0, 4.5, 28, 32}, {1.0, 5.0, 24, 28}, {1.0, 5.0, 28, 32},
                                   {1.2, 4.5, 16, 24}, {1.2, 4.5, 20, 28}, {1.0, 4.5, 20, 28}};
  const int M = (N - 1) / 2;
  std::vector<cplx> al, b;
  for (const auto& c : cand) {
    const double X = c[0] * M - c[3];
    if (X < 8.0) continue;
    double r = 0;
    if (wide_candidate(X, delta, c[0], c[1], (int)c[2], c[3], al, b, &r) && (int)al.size() == N) {
      store(al, b, r, X, c[1] * c[0], c[0], out, (int)c[2]);
      return EO_OK;
    }
  }
  return fail(EO_ERR_FIT, "no admissible rational approximant for this pole count");
}

// Index (s-major over the spacings ss, then the sigma/s ratios rs) of the first grid
// candidate whose N-pole line fits band X, or -1.  The candidates are evaluated in parallel
// host threads; the first in grid order is kept, so the result does not depend on threads.
static int first_accepted(int N, double X, double delta, const double* ss, int ns_, const double* rs, int nr) {
  const int M = (N - 1) / 2;
  const int nc = ns_ * nr;
  std::vector<char> ok(nc, 0);
  std::atomic<int> next(0);
  auto work = [&] {
    std::vector<cplx> al, b;
    for (int ci = next++; ci < nc; ci = next++) {
      const double sp = ss[ci / nr], ratio = rs[ci % nr];
      double r;
      if (sp * M >= X && residues(N, ratio * sp, sp, X, al, b) && accept(X, delta, al, b, &r)) ok[ci] = 1;
    }
  };
  const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) th.emplace_back(work);
  for (auto& x : th) x.join();
  for (int ci = 0; ci < nc; ++ci)
    if (ok[ci]) return ci;
  return -1;
}

eo_status fit_for_band(double X, double delta, int nmax, Fit& out) {
  if (!(X > 0)) return fail(EO_ERR_INVALID_ARG, "band*tau must be positive");
  if (X > 40.0) return fit_wide(X, delta, out);
  // fewest poles: the coarse search grid first, then the fine one, then the wide
  // construction (trapezoidal centre, fitted ends), which needs more poles
  const double* grids[2][2] = {{kS, kRatio}, {kSFine, kRatioFine}};
  const int sizes[2][2] = {{(int)(sizeof(kS) / sizeof(kS[0])), (int)(sizeof(kRatio) / sizeof(kRatio[0]))},
                           {(int)(sizeof(kSFine) / sizeof(kSFine[0])),
                            (int)(sizeof(kRatioFine) / sizeof(kRatioFine[0]))}};
  for (int gi = 0; gi < 2; ++gi) {
    for (int N = 5; N <= std::min(nmax, 101); N += 2) {
      const int ci = first_accepted(N, X, delta, grids[gi][0], sizes[gi][0], grids[gi][1], sizes[gi][1]);
      if (ci < 0) continue;
      const double sp = grids[gi][0][ci / sizes[gi][1]], ratio = grids[gi][1][ci % sizes[gi][1]];
      std::vector<cplx> al, b;
      double r;
      residues(N, ratio * sp, sp, X, al, b);
      accept(X, delta, al, b, &r);
      store(al, b, r, X, ratio * sp, sp, out);
      return EO_OK;
    }
  }
  if (fit_wide(X, delta, out) == EO_OK) return EO_OK;
  return fail(EO_ERR_FIT, "band*tau too wide for the supported pole counts");
}

// ---------------------------------------------------------------- the paper's construction
// Sections 3.1-3.2.  A function f with f^ supported in [-1/(2h), 1/(2h)] is a sum of
// shifted Gaussians, f(x) = sum_m c_m psi_h(x + m h), psi_h(x) = (4 pi)^{-1/2}
// e^{-x^2/(4h^2)}, c_m = h int e^{-2 pi i m h xi} f^(xi) / psi_h^(xi) dxi with
// psi_h^(xi) = h e^{-4 pi^2 h^2 xi^2}; for e^{2 pi i t x}, c_m = e^{4 pi^2 h^2 t^2}
// e^{-2 pi i m h t}.  Each psi_h(x + m h) = psi_1(x/h + m) is replaced by the Table 1
// rational psi_1(y) ~= Re sum_{j=-L..L} a_j / (i y + mu + i j).  For real x,
// Re w = (w + conj w)/2; in z = 2 pi i x (so z = i theta, e^z = e^{2 pi i x}) the two
// halves are two vertical pole lines, n = -(M+L)..M+L:
//   p+_n = -2 pi h (mu + i n)  (right half-plane, mu < 0),  residue  pi h sum_{m+j=n} c_m a_j,
//   p-_n =  2 pi h (mu - i n)  (its mirror image),          residue -pi h sum_{m+j=n} c_m conj(a_j).
// Table 1 is used through its even part (a_j + conj(a_{-j}))/2 (psi_1 is even, so the error
// does not grow), which makes the approximant exactly conjugate-closed.

// Table 1 (Section 3.2): mu and (Re a_j, Im a_j), j = -11..11.
static const int kTabL = 11;
static const double kTabMu = -4.315321510875024;
static const double kTabA[2 * kTabL + 1][2] = {
    {-1.0845749544592896e-7, 2.77075431662228e-8},  {1.858753344202957e-8, -9.105375434750162e-7},
    {3.6743713227243024e-6, 7.073284346322969e-7},  {-2.7990058083347696e-6, 0.0000112564827639346},
    {0.000014918577548849352, -0.0000316278486761932}, {-0.0010751767283285608, -0.00047282220513073084},
    {0.003816465653840016, 0.017839810396560574},  {0.12124105653274578, -0.12327042473830248},
    {-0.9774980792734348, -0.1877130220537587},    {1.3432866123333178, 3.2034715228495942},
    {4.072408546157305, -6.123755543580666},       {-9.442699917778205, 0.0},
    {4.072408620272648, 6.123755841848161},        {1.3432860877712938, -3.2034712658530275},
    {-0.9774985292598916, 0.18771238018072134},    {0.1212417070363373, 0.12326987628935386},
    {0.0038169724770333343, -0.017839242222443888}, {-0.0010756025812659208, 0.0004731874917343858},
    {0.000014713754789095218, 0.000031358475831136815}, {-2.659323898804944e-6, -0.000011341571201752273},
    {3.6970377676364553e-6, -6.517457477594937e-7}, {3.883933649142257e-9, 9.128496023863376e-7},
    {-1.0816457995911385e-7, -2.954309729192276e-8}};

void distinct_poles(const Fit& f, std::vector<int>& idx) {
  idx.clear();
  const std::vector<int> lines = f.lines.empty() ? std::vector<int>{f.N()} : f.lines;
  int s0 = 0;
  for (int n : lines) {
    const int K = (n - 1) / 2;
    for (int j = 0; j <= K; ++j) idx.push_back(s0 + K + j);
    s0 += n;
  }
}

static std::vector<cplx> table_even() {
  std::vector<cplx> a(2 * kTabL + 1);
  for (int j = -kTabL; j <= kTabL; ++j) {
    const cplx p(kTabA[j + kTabL][0], kTabA[j + kTabL][1]), q(kTabA[kTabL - j][0], kTabA[kTabL - j][1]);
    a[j + kTabL] = 0.5 * (p + std::conj(q));
  }
  a[kTabL] = a[kTabL].real();
  return a;
}

static void gauss_poles(int M, double h, std::vector<cplx>& al) {
  const int K = M + kTabL, n1 = 2 * K + 1;
  al.resize(2 * (size_t)n1);
  for (int n = -K; n <= K; ++n) {
    const int i = K - n;                   // increasing imaginary part along each line
    al[i] = -2.0 * M_PI * h * cplx(kTabMu, n);
    al[n1 + i] = 2.0 * M_PI * h * cplx(kTabMu, -n);
  }
}

// Residues on the two lines for Gaussian-sum coefficients c (m = -M..M, c_{-m} = conj c_m),
// made exactly conjugate-symmetric along each line.
static void gauss_residues(int M, double h, const std::vector<cplx>& c, std::vector<cplx>& b) {
  const std::vector<cplx> a = table_even();
  const int L = kTabL, K = M + L, n1 = 2 * K + 1;
  b.assign(2 * (size_t)n1, cplx(0, 0));
  for (int m = -M; m <= M; ++m)
    for (int j = -L; j <= L; ++j) {
      const int i = K - (m + j);
      b[i] += M_PI * h * c[m + M] * a[j + L];
      b[n1 + i] -= M_PI * h * c[m + M] * std::conj(a[j + L]);
    }
  for (int l = 0; l < 2; ++l) {
    cplx* bl = &b[(size_t)l * n1];
    for (int k = 1; k <= K; ++k) bl[K - k] = std::conj(bl[K + k]);
    bl[K] = bl[K].real();
  }
}

// c_m of e^{2 pi i t x} (eq. "coeff. for exp, gauss" with the normalisation of Section 3.1).
static void exp_coeffs(int M, double h, double t, std::vector<cplx>& c) {
  c.resize(2 * (size_t)M + 1);
  const double g = std::exp(4.0 * M_PI * M_PI * h * h * t * t);
  for (int m = 0; m <= M; ++m) {
    c[M + m] = g * std::exp(cplx(0.0, -2.0 * M_PI * m * h * t));
    c[M - m] = std::conj(c[M + m]);
  }
  c[M] = c[M].real();
}

// Gauss-Legendre nodes and weights on [0, 1] (Newton on the three-term recurrence).
static void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::abs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);   // 2/((1-z^2) P'^2), halved for [0, 1]
  }
}

// c_m of phi1(2 pi i x) = int_0^1 e^{2 pi i s x} ds: the integral over s of the
// exp coefficients, by composite 16-point Gauss-Legendre panels short enough for
// the oscillation e^{-2 pi i m h s} at |m| = M.
static void phi1_coeffs(int M, double h, std::vector<cplx>& c) {
  std::vector<double> gx, gw;
  gauss_legendre01(16, gx, gw);
  const int panels = std::max(4, (int)std::ceil(2.0 * M_PI * M * h / 2.0) + 1);
  c.assign(2 * (size_t)M + 1, cplx(0, 0));
  par_for(M + 1, [&](int64_t m0, int64_t m1) {
    for (int64_t m = m0; m < m1; ++m) {
      cplx acc(0, 0);
      for (int pnl = 0; pnl < panels; ++pnl)
        for (int k = 0; k < 16; ++k) {
          const double s = (pnl + gx[k]) / panels;
          acc += (gw[k] / panels) * std::exp(4.0 * M_PI * M_PI * h * h * s * s) *
                 std::exp(cplx(0.0, -2.0 * M_PI * m * h * s));
        }
      c[M + m] = acc;
    }
  });
  for (int m = 1; m <= M; ++m) c[M - m] = std::conj(c[M + m]);
  c[M] = c[M].real();
}

// c_m of phi2(2 pi i x) = int_0^1 (1 - s) e^{2 pi i s x} ds: the exp coefficients
// weighted by (1 - s) and integrated over s, by the same panels as phi1_coeffs.
static void phi2_coeffs(int M, double h, std::vector<cplx>& c) {
  std::vector<double> gx, gw;
  gauss_legendre01(16, gx, gw);
  const int panels = std::max(4, (int)std::ceil(2.0 * M_PI * M * h / 2.0) + 1);
  c.assign(2 * (size_t)M + 1, cplx(0, 0));
  par_for(M + 1, [&](int64_t m0, int64_t m1) {
    for (int64_t m = m0; m < m1; ++m) {
      cplx acc(0, 0);
      for (int pnl = 0; pnl < panels; ++pnl)
        for (int k = 0; k < 16; ++k) {
          const double s = (pnl + gx[k]) / panels;
          acc += (gw[k] / panels) * (1.0 - s) * std::exp(4.0 * M_PI * M_PI * h * h * s * s) *
                 std::exp(cplx(0.0, -2.0 * M_PI * m * h * s));
        }
      c[M + m] = acc;
    }
  });
  for (int m = 1; m <= M; ++m) c[M - m] = std::conj(c[M + m]);
  c[M] = c[M].real();
}

// phi1(z) = (e^z - 1) / z and phi2(z) = (e^z - 1 - z) / z^2 on z = i theta, by their
// Taylor series near 0 (where the closed forms cancel)
static cplx phi_value(int j, double th) {
  const cplx z(0.0, th);
  if (std::abs(th) < 0.5) {
    // sum_k z^k / (k + j)!, k = 0 .. 20 (remainder below 1e-25)
    cplx term = 1.0, acc = 0.0;
    double fact = j == 1 ? 1.0 : 2.0;   // j!
    for (int k = 0; k <= 20; ++k) {
      acc += term / fact;
      term *= z;
      fact *= (double)(k + j + 1);
    }
    return acc;
  }
  if (j == 1) return (std::exp(z) - 1.0) / z;
  return (std::exp(z) - 1.0 - z) / (z * z);
}

// max over theta in [t0, t1] (step dt) of |g(theta) - R(i theta)|.
static double band_err(const std::vector<cplx>& al, const std::vector<cplx>& b, double t0, double t1,
                       double dt, const std::function<cplx(double)>& g) {
  const int64_t n = std::max<int64_t>(2, (int64_t)std::ceil((t1 - t0) / dt) + 1);
  std::vector<double> part(64, 0.0);
  std::atomic<int> slot(0);
  par_for(n, [&](int64_t i0, int64_t i1) {
    double mx = 0;
    for (int64_t i = i0; i < i1; ++i) {
      const double th = t0 + (t1 - t0) * i / (n - 1);
      mx = std::max(mx, std::abs(g(th) - Reval(th, al, b)));
    }
    part[slot++] = mx;
  });
  return *std::max_element(part.begin(), part.end());
}

static void store_gauss(int M, double h, double X, const std::vector<cplx>& al, const std::vector<cplx>& b,
                        Fit& out) {
  const int N = (int)al.size(), n1 = N / 2;
  out.are.resize(N); out.aim.resize(N); out.bre.resize(N); out.bim.resize(N);
  for (int i = 0; i < N; ++i) {
    out.are[i] = al[i].real(); out.aim[i] = al[i].imag();
    out.bre[i] = b[i].real(); out.bim[i] = b[i].imag();
  }
  out.lines = {n1, n1};
  out.X = X; out.sigma = -2.0 * M_PI * h * kTabMu; out.s = 2.0 * M_PI * h; out.E = 0;
  out.gh = h; out.gM = M; out.gL = kTabL;
}

eo_status fit_gauss(double X, double h, double delta, Fit& out) {
  if (!(X > 0)) return fail(EO_ERR_INVALID_ARG, "band*tau must be positive");
  if (!(h > 0 && h < 0.5)) return fail(EO_ERR_INVALID_ARG, "Gaussian spacing h must be in (0, 0.5)");
  const int M0 = (int)std::ceil(X / (2.0 * M_PI * h));
  if (M0 > 400000) return fail(EO_ERR_INVALID_ARG, "band too wide for this spacing h");
  auto ex = [](double th) { return std::exp(cplx(0.0, th)); };
  std::vector<cplx> c, al, b;
  // R(-i theta) = conj R(i theta) exactly, so [0, X] suffices; the error grows
  // only near the ends of the Gaussian sum, so the edge window decides M.
  for (int M = M0; M <= M0 + 400; ++M) {
    exp_coeffs(M, h, 1.0, c);
    gauss_poles(M, h, al);
    gauss_residues(M, h, c, b);
    if (band_err(al, b, std::max(0.0, X - 40.0), X, 0.02, ex) > delta) continue;
    if (band_err(al, b, 0.0, X, 0.02, ex) > delta)
      return fail(EO_ERR_FIT, "Gaussian-sum approximant misses delta inside the band (h too large)");
    store_gauss(M, h, X, al, b, out);
    return EO_OK;
  }
  return fail(EO_ERR_FIT, "no Gaussian-sum approximant meets delta");
}

// Residues of exp(c z), phi1(z) or the partition of unity (kind 2, c the fraction
// of the Gaussians kept) on the poles of a Gaussian-sum fit.
static eo_status fit_function_gauss(const Fit& f, int kind, double c, std::vector<cplx>& b, double& err) {
  const int M = f.gM;
  const double h = f.gh, X = f.X;
  std::vector<cplx> cm, al;
  gauss_poles(M, h, al);
  std::function<cplx(double)> g;
  if (kind == 0) {
    exp_coeffs(M, h, c, cm);
    g = [c](double th) { return std::exp(cplx(0.0, c * th)); };
  } else if (kind == 1) {
    phi1_coeffs(M, h, cm);
    g = [](double th) { return phi_value(1, th); };
  } else if (kind == 3) {
    phi2_coeffs(M, h, cm);
    g = [](double th) { return phi_value(2, th); };
  } else {
    if (!(c > 0 && c <= 1)) return fail(EO_ERR_INVALID_ARG, "filter fraction must be in (0, 1]");
    const int M0 = (int)std::floor(c * M);
    cm.assign(2 * (size_t)M + 1, cplx(0, 0));
    for (int m = -M0; m <= M0; ++m) cm[m + M] = 1.0;
    // chi(x) = sum_{|m|<=M0} psi_h(x + m h), x = theta / (2 pi); terms beyond 40 h are < e^{-400}
    g = [M0, h](double th) {
      const double x = th / (2.0 * M_PI);
      const int lo = std::max(-M0, (int)std::floor(-x / h) - 40), hi = std::min(M0, (int)std::ceil(-x / h) + 40);
      double s = 0;
      for (int m = lo; m <= hi; ++m) {
        const double y = (x + m * h) / h;
        s += std::exp(-0.25 * y * y);
      }
      return cplx(s / std::sqrt(4.0 * M_PI), 0.0);
    };
  }
  gauss_residues(M, h, cm, b);
  err = band_err(al, b, 0.0, X, 0.02, g);
  return EO_OK;
}

// ---------------------------------------------------------------- other functions, same poles
// Values on the imaginary axis of the functions the same poles can carry
// (dense output and phi-functions, Section 1.2 remarks on reusing the solves):
//   kind 0: exp(c z), 0 < c <= 1;   kind 1: phi1(z) = (exp(z) - 1) / z;
//   kind 3: phi2(z) = (exp(z) - 1 - z) / z^2.
static cplx fn_value(int kind, double c, double th) {
  if (kind == 0) return std::exp(cplx(0.0, c * th));
  return phi_value(kind == 3 ? 2 : 1, th);
}

// Residues b of sum_m b_m / (z - alpha_m) on the poles of `f` for the function
// `kind` (parameter c).  Poles of a narrow fit: every residue by least squares on
// [0, X].  Poles of a wide fit: the central residues from the trapezoidal rule of
// the Cauchy integral of the function along the pole line (spacing s),
//   exp(c z):  b_m = -(s / 2 pi) exp(c alpha_m),
//   phi1(z):   b_m = -(s / 2 pi) (exp(alpha_m) - 1) / alpha_m  (the integral over c in [0, 1]),
//   phi2(z):   b_m = -(s / 2 pi) (exp(alpha_m) - 1 - alpha_m) / alpha_m^2,
// and the E outermost pairs by least squares, as for exp(z) itself.
// err: max |f(i x) - R(i x)| on [0, X] (both signs by conjugate symmetry).
eo_status fit_function(const Fit& f, int kind, double c, std::vector<cplx>& b, double& err) {
  if (kind < 0 || kind > 3) return fail(EO_ERR_INVALID_ARG, "unknown function kind");
  if (kind == 0 && !(c > 0 && c <= 1)) return fail(EO_ERR_INVALID_ARG, "c must be in (0, 1]");
  if (f.gh > 0) return fit_function_gauss(f, kind, c, b, err);
  if (kind == 2) return fail(EO_ERR_UNSUPPORTED, "the filter needs the Gaussian-sum fitter");
  const int N = f.N(), M = (N - 1) / 2;
  const double X = f.X, s = f.s;
  std::vector<cplx> al(N);
  for (int i = 0; i < N; ++i) al[i] = cplx(f.are[i], f.aim[i]);
  b.assign(N, cplx(0, 0));
  int E = f.E > 0 ? f.E : M;   // least-squares pairs beyond the centre
  if (f.E > 0) {
    for (int m = 0; m <= M; ++m) {
      const cplx a = al[m + M];
      const cplx fa = kind == 0 ? std::exp(c * a)
                                : (kind == 1 ? (std::exp(a) - 1.0) / a : (std::exp(a) - 1.0 - a) / (a * a));
      b[m + M] = -(s / (2 * M_PI)) * fa;
      b[M - m] = std::conj(b[m + M]);
    }
    b[M] = b[M].real();
  }
  // least squares for b_0 (narrow fits) and the E outer pairs
  const bool with_centre = f.E == 0;
  const int ns = (int)std::ceil(X * (with_centre ? 20.0 : 8.0)) + 41;
  const int rows = 2 * ns, cols = 2 * E + (with_centre ? 1 : 0);
  std::vector<double> A((size_t)rows * cols), t(rows), x;
  par_for(ns, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      const double th = X * i / (ns - 1);
      const cplx z(0.0, th);
      cplx rc(0, 0);
      if (!with_centre)
        for (int m = -(M - E); m <= M - E; ++m) rc += b[m + M] / (z - al[m + M]);
      const cplx tg = fn_value(kind, c, th) - rc;
      t[i] = tg.real();
      t[ns + i] = tg.imag();
      int col = 0;
      if (with_centre) {
        const cplx v = 1.0 / (z - al[M]);
        A[(size_t)col * rows + i] = v.real();
        A[(size_t)col * rows + ns + i] = v.imag();
        ++col;
      }
      for (int k = 0; k < E; ++k, col += 2) {
        const int mm = M - E + 1 + k;
        const cplx pp = 1.0 / (z - al[mm + M]), nn = 1.0 / (z - al[-mm + M]);
        const cplx c1 = pp + nn, c2 = cplx(0, 1) * (pp - nn);
        A[(size_t)col * rows + i] = c1.real();
        A[(size_t)col * rows + ns + i] = c1.imag();
        A[(size_t)(col + 1) * rows + i] = c2.real();
        A[(size_t)(col + 1) * rows + ns + i] = c2.imag();
      }
    }
  });
  std::vector<double> sc(cols);
  for (int j = 0; j < cols; ++j) {
    double s2 = 0;
    for (int i = 0; i < rows; ++i) s2 += A[(size_t)j * rows + i] * A[(size_t)j * rows + i];
    sc[j] = std::sqrt(s2);
    if (sc[j] == 0) return fail(EO_ERR_FIT, "degenerate least-squares column");
    for (int i = 0; i < rows; ++i) A[(size_t)j * rows + i] /= sc[j];
  }
  if (!lsq(A, t, rows, cols, x)) return fail(EO_ERR_FIT, "least squares failed");
  int col = 0;
  if (with_centre) { b[M] = x[0] / sc[0]; col = 1; }
  for (int k = 0; k < E; ++k, col += 2) {
    const int mm = M - E + 1 + k;
    b[mm + M] = cplx(x[col] / sc[col], x[col + 1] / sc[col + 1]);
    b[-mm + M] = std::conj(b[mm + M]);
  }
  const int64_t nb = (int64_t)std::ceil(X / 0.02) + 1;
  std::vector<double> part(64, 0.0);
  std::atomic<int> slot(0);
  par_for(nb, [&](int64_t i0, int64_t i1) {
    double mx = 0;
    for (int64_t i = i0; i < i1; ++i) {
      const double th = X * i / (nb - 1);
      mx = std::max(mx, std::abs(fn_value(kind, c, th) - Reval(th, al, b)));
    }
    part[slot++] = mx;
  });
  err = *std::max_element(part.begin(), part.end());
  return EO_OK;
}

}  // namespace eo
