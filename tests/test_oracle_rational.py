"""Pins of oracle.rational against what the paper prints and what the
mathematics fixes (Section 1.2, eqs. RM_prop1 / RM_prop2; Section 3.2, Table 1)."""
import os

import numpy as np
import pytest

from oracle import rational

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_psi_rational.txt")


def load_table1():
    mu, a = None, []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        if t[0] == "mu":
            mu = float(t[1])
        else:
            a.append(float(t[1]) + 1j * float(t[2]))
    return mu, np.array(a)


def test_table1_reproduces_gaussian_to_printed_accuracy():
    # Section 3.2: the Table 1 rational approximates psi_1 with L-inf error ~7e-13
    # on the whole real line.  A wrong sign of mu, a swapped j index or a
    # dropped term gives errors of order 1e-1 or worse.
    mu, a = load_table1()
    assert a.size == 23
    x = np.linspace(-60.0, 60.0, 240001)
    err = np.abs(rational.psi_rational(x, mu, a) - rational.gaussian_psi1(x)).max()
    assert 5e-13 < err < 7.5e-13
    # far tail: both sides are ~0
    assert abs(rational.psi_rational(np.array([1e4]), mu, a)[0]) < 1e-9


def test_R_eval_matches_partial_fractions_by_hand():
    # R(z) = sum b/(z - alpha): one pole, closed form; two poles combined into
    # a single fraction (b1 (z-a2) + b2 (z-a1)) / ((z-a1)(z-a2)).
    a = np.array([1.0 + 2.0j, 3.0 - 1.0j])
    b = np.array([0.5 - 1.0j, 2.0 + 0.25j])
    z = np.array([0.3j, -2.0 + 1.0j, 7.0])
    want = (b[0] * (z - a[1]) + b[1] * (z - a[0])) / ((z - a[0]) * (z - a[1]))
    assert np.allclose(rational.R_eval(z, a, b), want, rtol=1e-14, atol=0)


@pytest.mark.parametrize("n_poles", [21])
def test_own_fit_meets_contract(n_poles):
    alpha, b, X = rational.fit(n_poles, 1e-10, s_grid=[1.3, 1.4, 1.5], ratio_grid=(3.75, 4.0))
    band, mod, tail = rational.check_contract(alpha, b, X, 1e-10)
    assert X >= 3.0
    assert band <= 1e-10
    assert mod <= 1.0 + 1e-12
    assert tail < 1.0
    # conjugate-closed: b_{-m} = conj(b_m), alpha_{-m} = conj(alpha_m)
    assert np.array_equal(alpha[::-1], np.conj(alpha))
    assert np.array_equal(b[::-1], np.conj(b))
    # R(z) with such (alpha, b) is real on the real axis
    zr = np.linspace(-5, 5, 11) + 0j
    assert np.abs(rational.R_eval(zr, alpha, b).imag).max() < 1e-12 * np.abs(b).sum()


def test_check_contract_detects_violation():
    # a pole pair moved onto the imaginary axis side makes |R| blow up near it
    alpha, b, X = rational.fit(21, 1e-10, s_grid=[1.4], ratio_grid=(3.75,))
    bad_b = b.copy()
    bad_b[0] *= 1.001
    band, mod, _ = rational.check_contract(alpha, bad_b, X, 1e-10)
    assert band > 1e-10 or mod > 1.0 + 1e-12
