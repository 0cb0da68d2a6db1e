"""Pins of the oracle's restatement of the paper's own approximant
(``oracle/gauss.py``: Sections 3.1-3.3), each against something other than the
code under test: numerical Fourier integrals, Poisson summation, the closed forms
of e^{2 pi i x} and phi1, the Table 1 rational evaluated term by term, and the
paper's statements about the construction (two conjugate-closed pole lines, the
modulus exceeding one near |x| = M h, the filter bringing it back under one)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import gauss, rational
from oracle.resolvent import conjugate_closed
from tests.test_oracle_rational import load_table1

MU, A = load_table1()
pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


@pytest.mark.parametrize("h", [0.18, 0.3, 1.0])
@pytest.mark.parametrize("xi", [0.0, 0.5, 1.0, 1.7])
def test_psi_hat_is_the_fourier_transform(h, xi):
    # psi_h is even, so its transform is the cosine integral (numerical quadrature)
    val, _ = integrate.quad(lambda x: gauss.psi_h(x, h) * np.cos(2 * np.pi * x * xi), -40 * h, 40 * h,
                            limit=400, epsabs=1e-15, epsrel=1e-13)
    assert abs(val - gauss.psi_h_hat(xi, h)) <= 1e-13 * max(1.0, abs(val))


@pytest.mark.parametrize("h", [0.12, 0.18, 0.2])
def test_partition_of_unity_by_poisson_summation(h):
    # sum over all m of psi_h(x + m h) = psi_h^(0) / h = 1 up to e^{-4 pi^2} aliasing
    x = np.linspace(-3, 3, 1001)
    full = gauss.gauss_sum(x, np.ones(2 * 400 + 1, dtype=complex), h)
    assert np.abs(full - 1).max() <= 1e-14
    # the truncated window stays under one and falls to zero past M0 h (Section 3.3)
    M0 = 60
    chi = gauss.gauss_sum(np.linspace(-30, 30, 6001), gauss.window_coeffs(100, M0), h).real
    assert chi.max() <= 1.0 + 1e-14
    far = gauss.gauss_sum(np.array([(M0 + 15) * h, -(M0 + 15) * h]), gauss.window_coeffs(100, M0), h)
    assert np.abs(far).max() < 1e-10


@pytest.mark.parametrize("h,M", [(0.18, 160), (0.12, 120)])
def test_gaussian_sum_of_exp_meets_its_bound(h, M):
    c = gauss.exp_coeffs(M, h)
    x = np.linspace(-(M + 5) * h, (M + 5) * h, 8001)
    err = np.abs(gauss.gauss_sum(x, c, h) - np.exp(2j * np.pi * x))
    bound = gauss.alias_bound(x, M, h)
    # slack: the phases 2 pi m h of the coefficients carry ~|m| eps of rounding
    assert np.all(err <= bound + 1e-13)
    inside = np.abs(x) <= (M - 10) * h
    assert err[inside].max() <= 1e-10
    # the truncation shows at the ends of the sum
    assert err[~inside].max() > 1e-3


def test_exp_coefficients_for_other_times():
    # e^{2 pi i t x} for t = 0.5: the same Gaussians, only the coefficients change
    h, M = 0.18, 120
    x = np.linspace(-(M - 10) * h, (M - 10) * h, 4001)
    err = np.abs(gauss.gauss_sum(x, gauss.exp_coeffs(M, h, 0.5), h) - np.exp(1j * np.pi * x))
    assert err.max() <= 1e-10


def test_phi1_coefficients():
    h, M = 0.18, 120
    x = np.linspace(-(M - 10) * h, (M - 10) * h, 4001)
    x = x[np.abs(x) > 1e-9]
    want = (np.exp(2j * np.pi * x) - 1) / (2j * np.pi * x)
    err = np.abs(gauss.gauss_sum(x, gauss.phi1_coeffs(M, h), h) - want)
    assert err.max() <= 1e-10


def test_phi2_coefficients():
    # phi2(z) = (e^z - 1 - z) / z^2 at z = 2 pi i x; near 0 by its series 1/2 + z/6 + z^2/24
    h, M = 0.18, 120
    x = np.linspace(-(M - 10) * h, (M - 10) * h, 4001)
    z = 2j * np.pi * x
    want = np.where(np.abs(z) > 1e-3, (np.exp(z) - 1 - z) / np.where(z == 0, 1, z) ** 2,
                    0.5 + z / 6 + z * z / 24 + z ** 3 / 120)
    err = np.abs(gauss.gauss_sum(x, gauss.phi2_coeffs(M, h), h) - want)
    assert err.max() <= 1e-10
    # a plausible slip (the phi1 weight) is caught
    err1 = np.abs(gauss.gauss_sum(x, gauss.phi1_coeffs(M, h), h) - want)
    assert err1.max() > 0.1


def test_even_table_is_no_worse_and_conjugate_symmetric():
    ae = gauss.even_table(A)
    assert np.array_equal(ae[::-1], np.conj(ae))
    x = np.linspace(-60, 60, 120001)
    e_raw = np.abs(rational.psi_rational(x, MU, A) - rational.gaussian_psi1(x)).max()
    e_even = np.abs(rational.psi_rational(x, MU, ae) - rational.gaussian_psi1(x)).max()
    assert e_even <= e_raw * (1 + 1e-3) and e_even < 7.2e-13


@pytest.mark.parametrize("table", ["even", "printed"])
def test_composed_rational_equals_the_gaussian_sum_of_table1_rationals(table):
    # R(2 pi i x) against sum_m c_m psi_rational(x/h + m), the Table 1 rational
    # evaluated term by term: checks both pole lines, the residue bookkeeping and
    # the mirror terms of Re
    a = gauss.even_table(A) if table == "even" else A
    h, M = 0.18, 40
    c = gauss.exp_coeffs(M, h)
    alpha, b = gauss.compose(c, h, MU, a)
    rng = np.random.default_rng(5)
    x = rng.uniform(-(M + 8) * h, (M + 8) * h, 400)
    direct = sum(c[m + M] * rational.psi_rational(x / h + m, MU, a) for m in range(-M, M + 1))
    R = rational.R_eval(2j * np.pi * x, alpha, b)
    assert np.abs(R - direct).max() <= 1e-13 * np.abs(direct).max()


def test_pole_lines_and_conjugate_closure():
    h, M = 0.18, 30
    alpha, b = gauss.compose(gauss.exp_coeffs(M, h), h, MU, gauss.even_table(A))
    K = M + 11
    n1 = 2 * K + 1
    assert alpha.size == 2 * n1
    right, left = alpha[:n1], alpha[n1:]
    assert np.allclose(right.real, -2 * np.pi * h * MU) and -2 * np.pi * h * MU > 0
    assert np.allclose(left, -np.conj(right))                 # mirror image in the imaginary axis
    assert np.all(np.diff(right.imag) > 0) and np.all(np.diff(left.imag) > 0)
    assert conjugate_closed(alpha, b, tol=1e-13 * np.abs(b).max())


def test_h_018_covers_27_3_at_1e_10_with_690_poles():
    # h = 0.18 covers |x| <= 27.3 (|theta| <= 2 pi 27.3) at 1e-10 with M = 161:
    # 2 lines x (2 (M + 11) + 1) = 690 poles (M = 160 gives 686 poles at 3.5e-10)
    X = 2 * np.pi * 27.3
    alpha, b, M = gauss.gauss_fit(X, 0.18, MU, A)
    assert M == 161 and alpha.size == 690
    assert gauss.band_error(alpha, b, X) <= 1e-10
    a160, b160 = gauss.compose(gauss.exp_coeffs(160, 0.18), 0.18, MU, gauss.even_table(A))
    assert a160.size == 686 and 1e-10 < gauss.band_error(a160, b160, X) < 1e-9


def test_modulus_exceeds_one_near_the_ends_and_the_filter_fixes_it():
    # Section 3.3: the Gaussian approximant has |R| > 1 near |x| ~ M h; with the
    # partition-of-unity filter S (kept fraction M0 < M) |S R| <= 1 on the whole axis
    h = 0.18
    X = 2 * np.pi * 27.3
    alpha, b, M = gauss.gauss_fit(X, h, MU, A)
    y = np.linspace(-2 * np.pi * (M * h + 30), 2 * np.pi * (M * h + 30), 100001)
    R = rational.R_eval(1j * y, alpha, b)
    top = np.argmax(np.abs(R))
    assert np.abs(R).max() > 1.3
    assert abs(abs(y[top]) / (2 * np.pi) - M * h) < 2.0
    M0 = M - 12
    bq = gauss.filter_residues(M, M0, h, MU, A)
    Q = rational.R_eval(1j * y, alpha, bq)
    assert np.abs(Q * R).max() <= 1.0 + 1e-9
    assert np.abs(Q).max() <= 1.0 + 1e-9
    # and S R still approximates e^{i theta} where the filter is flat
    inside = np.abs(y) <= 2 * np.pi * (M0 - 10) * h
    assert np.abs(Q[inside] * R[inside] - np.exp(1j * y[inside])).max() <= 3e-10
    # beyond the window the filtered step damps
    outside = np.abs(y) >= 2 * np.pi * (M0 + 12) * h
    assert np.abs(Q[outside] * R[outside]).max() < 1e-6
