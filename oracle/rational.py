"""Rational approximants R(z) = sum_m b_m / (z - alpha_m) of e^z on the
imaginary axis (Section 1.2, eqs. def_RM, RM_prop1, RM_prop2), written plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The oracle's own fit (used by its self-checks) puts the 2M+1 poles on one
conjugate-closed vertical line in the right half-plane, alpha_m = sigma + i s m,
m = -M..M, and finds the residues by linear least squares on samples of
e^{i theta}, theta in [-X, X], in the real basis that forces
b_{-m} = conj(b_m) (so R maps the real axis symmetrically and eq.
"conjugate, matrix inverses" of Section 3.3 can be used).  The paper builds its
poles from Gaussian sums (Section 3.1) and the 23-pole rational of Table 1
(Section 3.2); ``psi_rational`` evaluates that table so that tests can pin the
evaluation against the paper's printed accuracy.

Acceptance of any (alpha, b), whoever produced it, is ``check_contract``:
brute-force evaluation of eq. RM_prop1 on [-X, X] and of eq. RM_prop2 on a wide
grid of the real axis plus an analytic tail bound beyond it.
"""
from __future__ import annotations

import numpy as np


def R_eval(z, alpha, b):
    """R(z) = sum_m b_m / (z - alpha_m) for an array of complex z (eq. def_RM)."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.zeros(z.shape, dtype=np.complex128)
    zf = z.ravel()
    of = out.ravel()
    for i in range(0, zf.size, 2048):
        zz = zf[i:i + 2048]
        of[i:i + 2048] = (b[None, :] / (zz[:, None] - alpha[None, :])).sum(axis=1)
    return of.reshape(z.shape)


def pole_line(n_poles: int, sigma: float, s: float) -> np.ndarray:
    """alpha_m = sigma + i s m, m = -M..M (n_poles = 2M+1), in that order."""
    if n_poles % 2 != 1:
        raise ValueError("n_poles must be odd")
    M = (n_poles - 1) // 2
    return sigma + 1j * s * np.arange(-M, M + 1)


def fit_residues(alpha: np.ndarray, X: float, samples_per_unit: float = 20.0) -> np.ndarray:
    """Least-squares residues for poles alpha (ordered m = -M..M, conjugate
    pairs alpha_{-m} = conj(alpha_m)) so that R(i theta) ~ e^{i theta} on [-X, X].

    Unknowns: b_0 real and Re/Im of b_m, m = 1..M, with b_{-m} = conj(b_m).
    Because R(-i theta) = conj(R(i theta)) for such b, the samples are taken on
    [0, X] only; real and imaginary parts of the residual are separate rows.
    """
    N = alpha.size
    M = (N - 1) // 2
    th = np.linspace(0.0, X, int(np.ceil(X * samples_per_unit)) + 41)
    A = 1.0 / (1j * th[:, None] - alpha[None, :])            # samples x N
    cols = [A[:, M]]
    for k in range(1, M + 1):
        cols.append(A[:, M + k] + A[:, M - k])                 # coefficient of Re b_k
        cols.append(1j * (A[:, M + k] - A[:, M - k]))          # coefficient of Im b_k
    B = np.array(cols).T
    t = np.exp(1j * th)
    Br = np.vstack([B.real, B.imag])
    tr = np.concatenate([t.real, t.imag])
    scale = np.linalg.norm(Br, axis=0)
    x = np.linalg.lstsq(Br / scale, tr, rcond=None)[0] / scale
    b = np.zeros(N, dtype=np.complex128)
    b[M] = x[0]
    for k in range(1, M + 1):
        b[M + k] = x[2 * k - 1] + 1j * x[2 * k]
        b[M - k] = np.conj(b[M + k])
    return b


def check_contract(alpha, b, X: float, delta: float, n_band: int = 4001):
    """Brute-force check of eqs. RM_prop1 and RM_prop2.

    Returns (band_error, max_modulus, tail_bound): band_error is
    max |e^{i theta} - R(i theta)| on a grid of [-X, X]; max_modulus is
    max |R(i y)| on a grid of |y| <= Y with spacing <= 0.02 and Y well beyond
    every pole; tail_bound bounds |R(i y)| for |y| > Y by sum|b| / (|y| - max|alpha|).
    """
    alpha = np.asarray(alpha)
    b = np.asarray(b)
    th = np.linspace(-X, X, n_band)
    band = np.abs(np.exp(1j * th) - R_eval(1j * th, alpha, b)).max()
    amax = np.abs(alpha).max()
    Y = max(50.0 * X + 200.0, 4.0 * amax + 200.0, amax + 2.0 * np.abs(b).sum())
    y = np.linspace(-Y, Y, int(2 * Y / 0.02) + 1)
    mod = np.abs(R_eval(1j * y, alpha, b)).max()
    tail = np.abs(b).sum() / (Y - amax)
    return band, mod, tail


def fit(n_poles: int, delta: float = 1e-10, s_grid=None, ratio_grid=None, X_step=0.25,
        bmax: float = 100.0):
    """The oracle's own fit for a given pole count: search (s, sigma/s, X) and
    keep the widest band X whose least-squares fit meets eq. RM_prop1 at delta
    and eq. RM_prop2 (after dividing b by max|R| when that exceeds 1 by less
    than delta / 10), with every |b_m| <= bmax (large residues cancel in the
    pole sum and amplify rounding).  Returns (alpha, b, X)."""
    M = (n_poles - 1) // 2
    s_grid = s_grid if s_grid is not None else np.arange(0.8, 1.61, 0.1)
    ratio_grid = ratio_grid if ratio_grid is not None else (3.75, 4.0, 4.5, 5.0)
    best = None
    for s in s_grid:
        for ratio in ratio_grid:
            alpha = pole_line(n_poles, ratio * s, s)
            X = s * M
            while X > 0.5:
                b = fit_residues(alpha, X)
                th = np.linspace(0, X, 1501)
                e = np.abs(np.exp(1j * th) - R_eval(1j * th, alpha, b)).max()
                if e <= 0.5 * delta and np.abs(b).max() <= bmax:
                    y = np.linspace(0, 50 * X + 200, 40001)
                    r = np.abs(R_eval(1j * y, alpha, b)).max()
                    if r <= 1 + 0.1 * delta:
                        if best is None or X > best[2]:
                            best = (alpha, b / max(r, 1.0), X)
                        break
                X -= X_step
    if best is None:
        raise RuntimeError("no admissible fit")
    return best


# --------------------------------------------------------------- Table 1

def psi_rational(x, mu: float, a: np.ndarray) -> np.ndarray:
    """R(x) = Re sum_{j=-L}^{L} a_j / (i x + mu + i j) with a = a_{-L..L}
    (eq. "approx of Gaussian via rationals", Section 3.2)."""
    L = (len(a) - 1) // 2
    j = np.arange(-L, L + 1)
    x = np.asarray(x, dtype=np.float64)
    den = 1j * x[..., None] + mu + 1j * j
    return (a / den).sum(axis=-1).real


def gaussian_psi1(x):
    """psi_1(x) = (4 pi)^{-1/2} exp(-x^2 / 4) (Section 3)."""
    return np.exp(-np.asarray(x) ** 2 / 4.0) / np.sqrt(4.0 * np.pi)
