"""The paper's own construction of the rational approximant (Sections 1.2, 3.1,
3.2, 3.3): a sum of shifted Gaussians, each Gaussian replaced by the rational of
Table 1, and the rational partition of unity used as a filter.  Written
plainly, in the paper's order, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation (Section 1.2 and Section 3.1):
  psi_h(x)      = (4 pi)^{-1/2} exp(-x^2 / (4 h^2)),
  psi_h^(xi)    = h exp(-4 pi^2 h^2 xi^2)      (its Fourier transform,
                                                 f^(xi) = int f(x) e^{-2 pi i x xi} dx),
  f(x)         ~= sum_{m=-M..M} c_m psi_h(x + m h)                   (Section 3.1),
  c_m           = h int e^{-2 pi i m h xi} f^(xi) / psi_h^(xi) dxi,
  e^{2 pi i t x}: c_m = h e^{-2 pi i m h t} / psi_h^(t)   (eq. "coeff. for exp, gauss"),
  psi_1(x)     ~= Re sum_{j=-L..L} a_j / (i x + mu + i j)  (eq. "approx of Gaussian via
                                                 rationals", Table 1: L = 11).

The approximant of e^z on z = i theta uses x = theta / (2 pi), so
e^{i theta} = e^{2 pi i x}.  Replacing every psi_h(x + m h) = psi_1(x/h + m) by
the Table 1 rational and writing Re w = (w + conj w) / 2 for real x gives a
rational function of z = 2 pi i x with two vertical pole lines (Section 3.3
speaks of the poles as complex-conjugate pairs; the mirror line comes from the
conjugate half of Re):
  p+_n = -2 pi h (mu + i n),          b+_n =  pi h sum_{m+j=n} c_m a_j,
  p-_n =  2 pi h (mu - i n),          b-_n = -pi h sum_{m+j=n} c_m conj(a_j),
n = -(M+L)..(M+L).  With mu < 0 the first line lies in the right half-plane and
the second is its mirror image in the imaginary axis.

Readings (where the paper is garbled or silent):
  * Section 1.2 prints c_m = (psi_h^(1)/h) e^{-2 pi i n h} and a "2 Re" form
    with poles at ix = mu + ij; Section 3.1 derives c_m = h e^{-2 pi i m h} /
    psi_h^(1), and the Table 1 coefficients reproduce psi_1 to the printed
    7e-13 only in the Section 3.2 form with factor 1.  We take Section 3.1 and
    Section 3.2.
  * Table 1's a_{-j} and conj(a_j) differ in the 8th digit.  We use the even
    part of the Table 1 rational, a_j <- (a_j + conj(a_{-j})) / 2: psi_1 is
    even, so the error of the even part is at most that of the printed
    rational, and the approximant becomes exactly conjugate-closed
    (b at conj(p) equals conj(b at p)), as the conjugate-pole form of
    Section 3.3 requires.
  * Section 3.3 normalises the partition of unity by psi_h^(1); by Poisson
    summation sum_m psi_h(x + m h) = psi_h^(0)/h + O(e^{-4 pi^2}) = 1, so the
    window chi(x) = sum_{|m|<=M0} psi_h(x + m h) needs no factor.
  * The reduction algorithm of Section 3.3 (and of Section 1.2) is not given;
    the filter is used unreduced.  Its poles are then a subset of the
    approximant's (M0 <= M), so S(tau L) reuses the same resolvents.
"""
from __future__ import annotations

import numpy as np

from .rational import R_eval


def psi_h(x, h: float):
    """psi_h(x) = (4 pi)^{-1/2} exp(-x^2 / (4 h^2)) (Section 1.2)."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(-x * x / (4.0 * h * h)) / np.sqrt(4.0 * np.pi)


def psi_h_hat(xi, h: float):
    """Fourier transform of psi_h: h exp(-4 pi^2 h^2 xi^2)."""
    xi = np.asarray(xi, dtype=np.float64)
    return h * np.exp(-4.0 * np.pi ** 2 * h * h * xi * xi)


# ------------------------------------------------------- Section 3.1 coefficients

def exp_coeffs(M: int, h: float, t: float = 1.0) -> np.ndarray:
    """c_m, m = -M..M, of e^{2 pi i t x} = sum c_m psi_h(x + m h):
    c_m = h e^{-2 pi i m h t} / psi_h^(t)  (eq. "coeff. for exp, gauss")."""
    m = np.arange(-M, M + 1)
    return h * np.exp(-2j * np.pi * m * h * t) / psi_h_hat(t, h)


def phi1_coeffs(M: int, h: float, n_quad: int = 400) -> np.ndarray:
    """c_m of phi1(2 pi i x) = (e^{2 pi i x} - 1) / (2 pi i x) = int_0^1 e^{2 pi i s x} ds:
    by linearity c_m = int_0^1 h e^{-2 pi i m h s} / psi_h^(s) ds, here by
    Gauss-Legendre quadrature in s (Section 3.1, the phi-function remark)."""
    s, w = np.polynomial.legendre.leggauss(n_quad)
    s = 0.5 * (s + 1.0)
    w = 0.5 * w
    m = np.arange(-M, M + 1)
    c = np.zeros(2 * M + 1, dtype=np.complex128)
    for k in range(n_quad):
        c += w[k] * h * np.exp(-2j * np.pi * m * h * s[k]) / psi_h_hat(s[k], h)
    return c


def phi2_coeffs(M: int, h: float, n_quad: int = 400) -> np.ndarray:
    """c_m of phi2(2 pi i x) = (e^{2 pi i x} - 1 - 2 pi i x) / (2 pi i x)^2
    = int_0^1 (1 - s) e^{2 pi i s x} ds: the exp coefficients weighted by (1 - s),
    integrated over s by Gauss-Legendre quadrature (Section 3.1, the phi-functions)."""
    s, w = np.polynomial.legendre.leggauss(n_quad)
    s = 0.5 * (s + 1.0)
    w = 0.5 * w
    m = np.arange(-M, M + 1)
    c = np.zeros(2 * M + 1, dtype=np.complex128)
    for k in range(n_quad):
        c += w[k] * (1.0 - s[k]) * h * np.exp(-2j * np.pi * m * h * s[k]) / psi_h_hat(s[k], h)
    return c


def window_coeffs(M: int, M0: int) -> np.ndarray:
    """c_m of the partition of unity chi(x) = sum_{|m|<=M0} psi_h(x + m h)
    (eq. "partition of unity-1"), embedded in m = -M..M."""
    m = np.arange(-M, M + 1)
    return (np.abs(m) <= M0).astype(np.complex128)


def gauss_sum(x, c: np.ndarray, h: float) -> np.ndarray:
    """sum_{m=-M..M} c_m psi_h(x + m h) for real x (Section 3.1)."""
    M = (c.size - 1) // 2
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape, dtype=np.complex128)
    for m in range(-M, M + 1):
        out += c[m + M] * psi_h(x + m * h, h)
    return out


def alias_bound(x, M: int, h: float) -> np.ndarray:
    """Right-hand side of eq. "error bound for e^ix, partial-1" for f = e^{2 pi i x},
    with the aliasing sum written out from Poisson summation:
    (h / psi_h^(1)) [ (1/h) sum_{k != 0} psi_h^(k/h + 1) + sum_{|m|>M} psi_h(x + m h) ]."""
    x = np.asarray(x, dtype=np.float64)
    alias = sum(psi_h_hat(k / h + 1.0, h) for k in range(-6, 7) if k != 0) / h
    tail = np.zeros(x.shape)
    for m in range(M + 1, M + 400):
        tail += psi_h(x + m * h, h) + psi_h(x - m * h, h)
    return (h / psi_h_hat(1.0, h)) * (alias + tail)


# ------------------------------------------------------- Section 3.2 / 3.3 rational

def even_table(a: np.ndarray) -> np.ndarray:
    """Even part of the Table 1 rational: a_j <- (a_j + conj(a_{-j})) / 2."""
    return 0.5 * (a + np.conj(a[::-1]))


def compose(c: np.ndarray, h: float, mu: float, a: np.ndarray):
    """Poles and residues of R(z) with R(2 pi i x) = sum_m c_m Re sum_j a_j /
    (i (x/h + m) + mu + i j): the Gaussian sum of Section 3.1 with every
    Gaussian replaced by the rational of Section 3.2.  Returns (alpha, b), the
    right line p+ (n = -(M+L)..M+L) followed by the mirror line p-, each in
    order of increasing imaginary part."""
    M = (c.size - 1) // 2
    L = (a.size - 1) // 2
    K = M + L
    bp = np.zeros(2 * K + 1, dtype=np.complex128)    # indexed by n + K
    bm = np.zeros(2 * K + 1, dtype=np.complex128)
    for m in range(-M, M + 1):
        for j in range(-L, L + 1):
            n = m + j
            bp[n + K] += np.pi * h * c[m + M] * a[j + L]
            bm[n + K] += -np.pi * h * c[m + M] * np.conj(a[j + L])
    n = np.arange(-K, K + 1)
    pp = -2.0 * np.pi * h * (mu + 1j * n)            # Im = -2 pi h n
    pm = 2.0 * np.pi * h * (mu - 1j * n)             # Im = -2 pi h n
    # order each line by increasing Im (n descending)
    alpha = np.concatenate([pp[::-1], pm[::-1]])
    b = np.concatenate([bp[::-1], bm[::-1]])
    return alpha, b


def band_error(alpha, b, X: float, t: float = 1.0, n: int = 20001) -> float:
    """max_{|theta|<=X} |e^{i t theta} - R(i theta)| on a uniform grid."""
    th = np.linspace(-X, X, n)
    return float(np.max(np.abs(np.exp(1j * t * th) - R_eval(1j * th, alpha, b))))


def gauss_fit(X: float, h: float, mu: float, a: np.ndarray, delta: float = 1e-10, M_max: int = 100000):
    """Smallest M whose composed approximant of e^z meets |e^{i theta} - R(i theta)|
    <= delta on [-X, X] (eq. RM_prop1); returns (alpha, b, M).  The search
    starts at the spatial half-width M h = X / (2 pi) (Section 1.2: valid for
    |x| up to about M h)."""
    ae = even_table(a)
    M = int(np.ceil(X / (2.0 * np.pi * h)))
    while M <= M_max:
        alpha, b = compose(exp_coeffs(M, h), h, mu, ae)
        if band_error(alpha, b, X, n=max(4001, int(40 * X) + 1)) <= delta:
            return alpha, b, M
        M += 1
    raise RuntimeError("no Gaussian-sum approximant within M_max")


def filter_residues(M: int, M0: int, h: float, mu: float, a: np.ndarray):
    """Residues of the unreduced rational partition of unity Q(z), Q(2 pi i x)
    ~= chi(x) (eq. "partition of unity"), on the poles of the M-term
    approximant (they vanish beyond n = +-(M0 + L))."""
    return compose(window_coeffs(M, M0), h, mu, even_table(a))[1]
