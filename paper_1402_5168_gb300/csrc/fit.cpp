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
  if (N > 101) return fit_wide_poles(N, delta, out);
  if (fit_for_poles_grid(N, delta, out, kS, (int)(sizeof(kS) / sizeof(kS[0])), kRatio,
                         (int)(sizeof(kRatio) / sizeof(kRatio[0]))) == EO_OK)
    return EO_OK;
  if (fit_for_poles_grid(N, delta, out, kSFine, (int)(sizeof(kSFine) / sizeof(kSFine[0])), kRatioFine,
                         (int)(sizeof(kRatioFine) / sizeof(kRatioFine[0]))) == EO_OK)
    return EO_OK;
  if (fit_wide_poles(N, delta, out) == EO_OK) return EO_OK;
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

eo_status fit_for_band(double X, double delta, int nmax, Fit& out) {
  if (!(X > 0)) return fail(EO_ERR_INVALID_ARG, "band*tau must be positive");
  if (X > 40.0) return fit_wide(X, delta, out);
  std::vector<cplx> al, b;
  for (int N = 5; N <= std::min(nmax, 301); N += 2) {
    const int M = (N - 1) / 2;
    for (double s : kS)
      for (double ratio : kRatio) {
        if (s * M < X) continue;
        double r;
        if (residues(N, ratio * s, s, X, al, b) && accept(X, delta, al, b, &r)) {
          store(al, b, r, X, ratio * s, s, out);
          return EO_OK;
        }
      }
  }
  return fail(EO_ERR_FIT, "band*tau too wide for the supported pole counts");
}

// ---------------------------------------------------------------- other functions, same poles
// Values on the imaginary axis of the functions the same poles can carry
// (dense output and phi-functions, Section 1.2 remarks on reusing the solves):
//   kind 0: exp(c z), 0 < c <= 1;   kind 1: phi1(z) = (exp(z) - 1) / z.
static cplx fn_value(int kind, double c, double th) {
  if (kind == 0) return std::exp(cplx(0.0, c * th));
  if (std::abs(th) < 1e-6) return cplx(1.0 - th * th / 6.0, th / 2.0 - th * th * th / 24.0);
  return (std::exp(cplx(0.0, th)) - 1.0) / cplx(0.0, th);
}

// Residues b of sum_m b_m / (z - alpha_m) on the poles of `f` for the function
// `kind` (parameter c).  Poles of a narrow fit: every residue by least squares on
// [0, X].  Poles of a wide fit: the central residues from the trapezoidal rule of
// the Cauchy integral of the function along the pole line (spacing s),
//   exp(c z):  b_m = -(s / 2 pi) exp(c alpha_m),
//   phi1(z):   b_m = -(s / 2 pi) (exp(alpha_m) - 1) / alpha_m  (the integral over c in [0, 1]),
// and the E outermost pairs by least squares, as for exp(z) itself.
// err: max |f(i x) - R(i x)| on [0, X] (both signs by conjugate symmetry).
eo_status fit_function(const Fit& f, int kind, double c, std::vector<cplx>& b, double& err) {
  if (kind != 0 && kind != 1) return fail(EO_ERR_INVALID_ARG, "unknown function kind");
  if (kind == 0 && !(c > 0 && c <= 1)) return fail(EO_ERR_INVALID_ARG, "c must be in (0, 1]");
  const int N = f.N(), M = (N - 1) / 2;
  const double X = f.X, s = f.s;
  std::vector<cplx> al(N);
  for (int i = 0; i < N; ++i) al[i] = cplx(f.are[i], f.aim[i]);
  b.assign(N, cplx(0, 0));
  int E = f.E > 0 ? f.E : M;   // least-squares pairs beyond the centre
  if (f.E > 0) {
    for (int m = 0; m <= M; ++m) {
      const cplx a = al[m + M];
      b[m + M] = kind == 0 ? -(s / (2 * M_PI)) * std::exp(c * a) : -(s / (2 * M_PI)) * (std::exp(a) - 1.0) / a;
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
