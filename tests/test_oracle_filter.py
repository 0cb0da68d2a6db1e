"""Pins of the oracle's S(k0 Delta) (Section 3.3; oracle/filter.py) against what the
mathematics fixes, independently of the filter's own code:

* the scalar identity behind the shifted-Laplacian form: on the real line,
  Re sum_upper 2 s alpha / (-y^2 - alpha^2) equals the window chi(y / 2 pi), evaluated as
  the plain Gaussian sum of Section 3.3;
* a Fourier mode of a periodic square, and a cosine mode (a Neumann eigenfunction) of a
  walled square, is multiplied by the window chi(sqrt(k0) |k| / 2 pi), evaluated as the
  plain Gaussian sum of Section 3.3 (not through the rational): 1 below the window's
  edge, 0 beyond it, the window's value in between;
  (to the collocation error of the mode, which grows with |k|);
* constants pass unchanged (chi(0) = 1), on both domains;
* the conjugate-pole form (upper poles, weight 2 per pair) equals the real part of the
  full pole sum (Section 3.3, eq. "conjugate, matrix inverses").

A dropped alpha_m factor, a sign error in the shift, a wrong k0 scaling, or Dirichlet
instead of Neumann wall rows fails one of these.
"""
import numpy as np
import pytest

from oracle import gauss, sem
from oracle.filter import LaplacianFilter
from tests.test_oracle_rational import load_table1

MU, A = load_table1()
H, M, M0 = 0.18, 30, 27


@pytest.fixture(scope="module")
def poles():
    alpha, _ = gauss.compose(gauss.exp_coeffs(M, H), H, MU, gauss.even_table(A))
    s = gauss.filter_residues(M, M0, H, MU, A)
    return alpha, s


def chi(x):
    return gauss.gauss_sum(np.atleast_1d(np.asarray(x, dtype=np.float64)), gauss.window_coeffs(M, M0), H).real[0]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def mode_tol(kk):
    # collocation error of a mode with |k| / 2 pi = kk on 4 leaves of p = 16 per unit
    return 1e-10 if kk <= 3.7 else 1e-6


def test_shifted_laplacian_form_equals_the_window(poles):
    alpha, s = poles
    up = (alpha.imag >= 0) & (s != 0)
    wt = np.where(alpha[up].imag == 0, 1.0, 2.0)
    y = np.linspace(0.0, 60.0, 3001)
    q = np.array([np.sum(wt * s[up] * alpha[up] / (-(t * t) - alpha[up] ** 2)).real for t in y])
    c = gauss.gauss_sum(y / (2 * np.pi), gauss.window_coeffs(M, M0), H).real
    e = float(np.abs(q - c).max())
    print(f"shifted-Laplacian form vs window on [0, 60]: {e:.2e}")
    assert e <= 1e-10
    assert c[0] > 1 - 1e-10 and c[-1] < 1e-10      # both ends of the window are on the grid


@pytest.mark.parametrize("k0", [1.0, 0.49])
def test_periodic_fourier_modes_are_scaled_by_the_window(poles, k0):
    g = sem.Grid(4, 4, 16, periodic=True)
    flt = LaplacianFilter(g, k0, *poles)
    edge = M0 * H / np.sqrt(k0)       # |k| / 2 pi at the window's edge
    seen = set()
    for k1, k2 in [(1, 0), (2, 2), (3, 2), (3, 4), (5, 5), (6, 4)]:
        kk = np.hypot(k1, k2)
        phi = np.cos(2 * np.pi * (k1 * g.x + k2 * g.y))
        want = chi(np.sqrt(k0) * kk)
        got = flt.apply(phi)
        e = float(np.abs(got - want * phi).max())
        print(f"periodic k0={k0} mode ({k1},{k2}) |k|/2pi={kk:.3f} (edge {edge:.2f}): "
              f"chi={want:.6f}, max deviation {e:.2e}")
        assert e <= mode_tol(kk), (k1, k2, e)
        seen.add("pass" if want > 1 - 1e-9 else "stop" if want < 1e-9 else "edge")
    assert seen == {"pass", "stop", "edge"} or k0 != 1.0


def test_walled_cosine_modes_are_scaled_by_the_window(poles):
    g = sem.Grid(4, 4, 16)
    flt = LaplacianFilter(g, 1.0, *poles)
    for k1, k2 in [(0, 0), (2, 0), (4, 6), (7, 6), (10, 8)]:
        kk = 0.5 * np.hypot(k1, k2)          # cos(pi k x): |k| / 2 pi = k / 2
        phi = np.cos(np.pi * k1 * g.x) * np.cos(np.pi * k2 * g.y)
        want = chi(kk)
        e = float(np.abs(flt.apply(phi) - want * phi).max())
        print(f"walls mode ({k1},{k2}) |k|/2pi={kk:.3f}: chi={want:.6f}, max deviation {e:.2e}")
        assert e <= mode_tol(kk), (k1, k2, e)


def test_constants_pass_and_pair_form_equals_full_sum(poles):
    for per in (True, False):
        g = sem.Grid(2, 2, 10, periodic=per)
        flt = LaplacianFilter(g, 1.0, *poles)
        one = np.ones(g.n_nodes)
        assert np.abs(flt.apply(one) - 1.0).max() <= 1e-9
        rng = np.random.default_rng(5)
        phi = rng.standard_normal(g.n_nodes)
        full = flt.apply_full(phi)
        assert np.abs(full.imag).max() <= 1e-9 * np.abs(full).max()
        assert rel(flt.apply(phi), full.real) <= 1e-12
