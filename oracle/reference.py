"""Independent references for the wave problem on small grids: the semi-discrete
operator L_h written as an explicit matrix, its exponential by dense
eigendecomposition, and classical RK4 with a tiny step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The collocation system of Section 2.2 fixes the interface values from the
interior ones (flux continuity) and the boundary values (u = 0), so the
semi-discrete wave operator acts on the interior unknowns only:
  u_e = E u_i,  E = -F_ee^{-1} F_ei      (flux rows at interface nodes)
  A_eff = A_ii + A_ie E                   (interior collocation rows)
  L_h (u_i, v_i) = (v_i, A_eff u_i).
Eq. "error in exp(t*L)" of Section 1.2 bounds |R(tau L_h) u - exp(tau L_h) u|
by delta |u| + 2 |u - P_Lambda u| (L_h is only approximately skew, Section 1.3).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .resolvent import Problem


class WaveLh:
    def __init__(self, prob: Problem):
        if prob.kind != "wave":
            raise ValueError("wave only")
        cls = prob.cls
        self.i = np.flatnonzero(cls == 0)
        self.e = np.flatnonzero(cls == 1)
        self.d = np.flatnonzero(cls == 2)
        A = prob.Lap.toarray()
        F = prob.Flux.toarray()
        Fee = F[np.ix_(self.e, self.e)]
        Fei = F[np.ix_(self.e, self.i)]
        self.E = -np.linalg.solve(Fee, Fei)
        self.Aeff = A[np.ix_(self.i, self.i)] + A[np.ix_(self.i, self.e)] @ self.E
        ni = self.i.size
        self.L = np.block([[np.zeros((ni, ni)), np.eye(ni)], [self.Aeff, np.zeros((ni, ni))]])
        self.n_nodes = prob.grid.n_nodes
        self._eig = None

    def lift(self, ui: np.ndarray, vi: np.ndarray) -> np.ndarray:
        """Full-node state on the constraint manifold from interior values."""
        u = np.zeros(self.n_nodes)
        v = np.zeros(self.n_nodes)
        u[self.i], v[self.i] = ui, vi
        u[self.e], v[self.e] = self.E @ ui, self.E @ vi
        return np.stack([u, v])

    def restrict(self, state: np.ndarray) -> np.ndarray:
        return np.concatenate([state[0][self.i], state[1][self.i]])

    def eig(self):
        if self._eig is None:
            lam, V = sla.eig(self.L)
            self._eig = (lam, V, np.linalg.inv(V))
        return self._eig

    def expm_apply(self, t: float, z: np.ndarray) -> np.ndarray:
        lam, V, Vi = self.eig()
        return (V @ (np.exp(t * lam) * (Vi @ z))).real

    def project_out(self, Lam: float, z: np.ndarray) -> np.ndarray:
        """z - P_Lambda z: the part of z on eigenvectors with |lambda| > Lambda."""
        lam, V, Vi = self.eig()
        c = Vi @ z
        c[np.abs(lam) <= Lam] = 0.0
        return (V @ c).real

    def rk4(self, t: float, z: np.ndarray, n: int) -> np.ndarray:
        dt = t / n
        L = self.L
        for _ in range(n):
            k1 = L @ z
            k2 = L @ (z + 0.5 * dt * k1)
            k3 = L @ (z + 0.5 * dt * k2)
            k4 = L @ (z + dt * k3)
            z = z + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        return z


def sw_fourier_exact(fields, x, y, t: float, f: float, g: float = 1.0, H: float = 1.0, n: int = 64):
    """Exact solution at time t of rotating shallow water u_t = f v - g h_x,
    v_t = -f u - g h_y, h_t = -H (u_x + v_y) on the periodic unit square, for
    band-limited initial fields, evaluated at the points (x, y).

    This is the exact reference of the paper's periodic shallow-water tests
    (Section 4.1): the operator is diagonalised in the Fourier domain.  Each
    field is given as a function of (X, Y); it is sampled on an n x n uniform grid
    of [0, 1)^2 (exact for trigonometric polynomials of degree < n/2), its Fourier
    coefficients are taken by FFT, every wavevector k evolves by exp(t M_k) with
    M_k = [[0, f, -i g k1], [-f, 0, -i g k2], [-i H k1, -i H k2, 0]] (the symbol
    of the operator, d/dx -> i k1), and the trigonometric sum is evaluated at the
    points.  Returns the stacked fields [u, v, h] at the points.
    """
    s = np.arange(n) / n
    X, Y = np.meshgrid(s, s, indexing="ij")
    hat = np.stack([np.fft.fft2(fn(X, Y)) / (n * n) for fn in fields])      # [3, n, n]
    kk = np.fft.fftfreq(n, d=1.0 / n)                                        # integer wavenumbers
    out = np.zeros((3, np.size(x)), dtype=np.complex128)
    xf = np.asarray(x, dtype=np.float64).ravel()
    yf = np.asarray(y, dtype=np.float64).ravel()
    for a in range(n):
        for b in range(n):
            c = hat[:, a, b]
            if np.max(np.abs(c)) < 1e-15:
                continue
            k1, k2 = 2 * np.pi * kk[a], 2 * np.pi * kk[b]
            M = np.array([[0, f, -1j * g * k1], [-f, 0, -1j * g * k2], [-1j * H * k1, -1j * H * k2, 0]])
            ct = sla.expm(t * M) @ c
            out += ct[:, None] * np.exp(1j * (k1 * xf + k2 * yf))[None, :]
    return out.real.reshape((3,) + np.shape(x))
