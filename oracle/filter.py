"""The filter S(k0 Delta) of Section 3.3 (the variant that follows the paper's
remark on the conjugate-pole shortcut): a rational partition of unity applied to
the Laplacian instead of to tau L, so that only the highest wavenumbers are damped.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Reading (the paper names the operator and says k0 follows from the initial data's
frequency content, nothing more).  The filter Q(z) = sum_m s_m / (z - alpha_m) of
Section 3.3 approximates the even window chi on the imaginary axis, Q(i theta) ~=
chi(theta / 2 pi).  With A = (-k0 Delta)^{1/2} (Delta <= 0), S(k0 Delta) := Q(i A):
a mode of wavenumber |k| (-Delta e = |k|^2 e) is multiplied by chi(sqrt(k0) |k| /
2 pi).  Because chi is even, Q(i A) = (Q(i A) + Q(-i A)) / 2 up to the fit error, and

    (i A - alpha)^{-1} + (-i A - alpha)^{-1} = -2 alpha (A^2 + alpha^2)^{-1},

so S(k0 Delta) = sum_m s_m alpha_m (k0 Delta - alpha_m^2)^{-1}: one shifted-Laplacian
solve per pole, no square root.  For a real field and conjugate-closed poles the sum
is the real part of the sum over the upper poles with weight 2 on each pair
(Section 3.3, eq. "conjugate, matrix inverses").  k0 is then chosen so that the
window's edge sqrt(k0) |k| = 2 pi M0 h lies above the wavenumbers the data carry.

Discretisation: the collocation Laplacian of Section 2.2 at interior nodes, flux
continuity on interfaces, and on walls the natural condition of the Laplacian,
d_n w = 0 (the recovered normal derivative), so that constants pass unchanged; a
periodic grid has no walls.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import sem


class LaplacianFilter:
    """S(k0 Delta) on a grid for the filter poles alpha and residues s."""

    def __init__(self, grid: sem.Grid, k0: float, alpha, s):
        self.grid = grid
        self.k0 = float(k0)
        self.alpha = np.asarray(alpha, dtype=np.complex128)
        self.s = np.asarray(s, dtype=np.complex128)
        self.cls, self.side = grid.classify()
        n = grid.n_nodes
        ones = np.ones(n)
        self.Lap = sem.divgrad_operator(grid, ones)
        self.Flux = sem.flux_continuity_rows(grid, ones)
        Gx, Gy = sem.wall_gradient_rows(grid)
        xw = sp.diags(((self.side == 1) | (self.side == 3)).astype(float))
        yw = sp.diags(((self.side == 0) | (self.side == 2)).astype(float))
        self.Wall = xw @ Gx + yw @ Gy          # normal derivative rows on the walls
        self.P_int = sp.diags((self.cls == 0).astype(float))
        self._lu = {}

    def system(self, a: complex) -> sp.csc_matrix:
        """Rows of (k0 Delta - a^2) w = rhs at interior nodes, flux rows, wall rows."""
        n = self.grid.n_nodes
        B = self.P_int @ (self.k0 * self.Lap - (a * a) * sp.identity(n)) + self.Flux.astype(np.complex128) \
            + self.Wall.astype(np.complex128)
        return sp.csc_matrix(B)

    def solve(self, i: int, phi: np.ndarray) -> np.ndarray:
        """(k0 Delta - alpha_i^2)^{-1} phi with the interior data phi (zero on the other rows)."""
        if i not in self._lu:
            self._lu[i] = spla.splu(self.system(self.alpha[i]))
        rhs = np.where(self.cls == 0, phi, 0.0).astype(np.complex128)
        return self._lu[i].solve(rhs)

    def apply_full(self, phi: np.ndarray) -> np.ndarray:
        """sum over every pole of s_m alpha_m (k0 Delta - alpha_m^2)^{-1} phi (complex)."""
        out = np.zeros(self.grid.n_nodes, dtype=np.complex128)
        for i in range(self.alpha.size):
            if self.s[i] != 0:
                out += self.s[i] * self.alpha[i] * self.solve(i, phi)
        return out

    def apply(self, phi: np.ndarray) -> np.ndarray:
        """The real field S(k0 Delta) phi: real part of the sum over the upper poles
        (Im alpha >= 0), weight 2 on each conjugate pair (Section 3.3)."""
        out = np.zeros(self.grid.n_nodes, dtype=np.complex128)
        for i in range(self.alpha.size):
            a = self.alpha[i]
            if a.imag < 0 or self.s[i] == 0:
                continue
            w = 1.0 if a.imag == 0 else 2.0
            out += w * self.s[i] * a * self.solve(i, phi)
        return out.real
