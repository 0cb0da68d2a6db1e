"""Resolvents (tau L - alpha)^{-1} through the elliptic reformulation
(Section 2.1) on the global collocation system B u = f (Section 2.2), and the
rational time step u <- sum_m b_m (tau L - alpha_m)^{-1} u (Section 1.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Two problem kinds (state layout [field][node], real, on the public node order):

wave  u_t = v, v_t = div(c^2 grad u) on the unit square, u = 0 on the boundary.
      (tau L - alpha)(U, V) = (f_u, f_v) gives U = (tau V - f_u) / alpha and
      [div(c^2 grad .) - (alpha/tau)^2] V = (alpha f_v + tau A f_u) / tau^2 with
      A = div(c^2 grad .), V = 0 on the boundary (u = 0 there for all time).
      As in Example 2 of Section 2.1 (eq. "v for inhomog, inverse") the elliptic
      unknown is the time derivative; the paper writes a three-field form, this
      is the same elimination in the two-field (u, v) form.

sw    linearised rotating shallow water u_t = f v - g h_x, v_t = -f u - g h_y,
      h_t = -H (u_x + v_y), no normal flow at the walls (Example 1 of
      Section 2.1, eqs. "inverse oper, RSW" to "elliptic solve, RSW", with
      gravity g and depth H written out).  With K = [[-alpha, tau f],
      [-tau f, -alpha]] and D = alpha^2 + tau^2 f^2:
        (U, V) = K^{-1} (F + tau g grad h),
        (Delta - D/(tau^2 g H)) h = D/(tau^2 g H alpha) r
                                    - (alpha div F + tau f curl F)/(tau g alpha),
      and U = 0 (x-walls) / V = 0 (y-walls) become the oblique conditions
        alpha h_x + tau f h_y = -(alpha F1 + tau f F2)/(tau g)   (x = 0, 1)
        alpha h_y - tau f h_x = (tau f F1 - alpha F2)/(tau g)    (y = 0, 1).

kappa the three-field wave form of Section 2.1, Example 2 (eq. "forward oper, inhom"):
      u_tt = kappa Delta u on a periodic square, state (w, z, v) = (u_x, u_y, u_t),
      w_t = v_x, z_t = v_y, v_t = kappa (w_x + z_y).  With the data scaled by tau
      (eqs. "operator for inhomog, inverse" to "v for inhomog, inverse" with
      alpha -> alpha / tau), (tau L - alpha)(W, Z, V) = (f_w, f_z, f_v) gives
        (Delta - alpha^2 / (tau^2 kappa)) V = alpha f_v / (tau^2 kappa) + (d_x f_w + d_y f_z) / tau,
        W = (tau V_x - f_w) / alpha,   Z = (tau V_y - f_z) / alpha
      (eq. "w and z eqns"), V_x, V_y the recovered node gradient.  kappa is given at
      the nodes (c2=kappa).

With consistent=True the interior rows carry the extra term (tau f / alpha) Curl(G h),
G the recovered node gradient of the post-map: the exact elimination of (U, V) for this
discretisation, where Curl(G h) does not vanish next to leaf edges.  The per-pole solves
are then resolvents of one discrete operator.

Every solve is a sparse direct solve (scipy splu) of the full global system.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import sem


class Problem:
    """A discretised problem: grid, kind and coefficients."""

    def __init__(self, grid: sem.Grid, kind: str, tau: float, c2=None,
                 f: float = 0.0, g: float = 1.0, H: float = 1.0, consistent: bool = False):
        if kind not in ("wave", "sw", "kappa"):
            raise ValueError(kind)
        if kind == "kappa" and not grid.periodic:
            raise ValueError("the three-field wave form is set on a periodic square")
        self.grid, self.kind, self.tau = grid, kind, float(tau)
        self.f, self.g, self.H = float(f), float(g), float(H)
        self.cls, self.side = grid.classify()
        n = grid.n_nodes
        if kind == "wave":
            self.a = np.asarray(c2, dtype=np.float64)
            self.n_fields = 2
        elif kind == "kappa":
            self.kappa = np.asarray(c2, dtype=np.float64)
            self.a = np.ones(n)
            self.n_fields = 3
        else:
            self.a = np.ones(n)
            self.n_fields = 3
        self.Lap = sem.divgrad_operator(grid, self.a)
        self.Flux = sem.flux_continuity_rows(grid, self.a)
        if kind == "sw":
            self.Gx, self.Gy = sem.wall_gradient_rows(grid)
        # consistent elimination (shallow water): keep the (tau f / alpha) Curl(G h)
        # term that the continuum drops (curl grad = 0) but this discretisation does not
        self.consistent = bool(consistent) and kind == "sw"
        if self.consistent:
            self.CG = sem.curl_of_gradient(grid)
        self.P_int = sp.diags((self.cls == 0).astype(float))
        self.P_ifc = sp.diags((self.cls == 1).astype(float))
        self.P_bnd = sp.diags((self.cls == 2).astype(float))

    # -------------------------------------------------------------- system
    def kappa2(self, alpha: complex):
        """The shift of the elliptic rows: a number, or for the kappa form one per node."""
        if self.kind == "wave":
            return (alpha / self.tau) ** 2
        if self.kind == "kappa":
            return (alpha / self.tau) ** 2 / self.kappa
        D = alpha * alpha + (self.tau * self.f) ** 2
        return D / (self.tau ** 2 * self.g * self.H)

    def system(self, alpha: complex) -> sp.csc_matrix:
        """Global matrix: interior collocation rows, interface flux rows,
        boundary rows (Dirichlet identity for wave, oblique condition for sw)."""
        k2 = self.kappa2(alpha)
        n = self.grid.n_nodes
        shift = sp.diags(k2 * np.ones(n)) if np.ndim(k2) else k2 * sp.identity(n)
        B = self.P_int @ (self.Lap - shift) + self.Flux.astype(np.complex128)
        if self.kind == "kappa":
            return sp.csc_matrix(B)
        if self.kind == "wave":
            B = B + self.P_bnd
        else:
            xw = sp.diags(((self.side == 1) | (self.side == 3)).astype(float))
            yw = sp.diags(((self.side == 0) | (self.side == 2)).astype(float))
            tf = self.tau * self.f
            B = B + xw @ (alpha * self.Gx + tf * self.Gy) + yw @ (alpha * self.Gy - tf * self.Gx)
            if self.consistent:
                B = B + (tf / alpha) * self.CG
        return sp.csc_matrix(B)

    def rhs(self, alpha: complex, state: np.ndarray) -> np.ndarray:
        """Right-hand side of the elliptic system for input state (the pre-map)."""
        tau = self.tau
        if self.kind == "wave":
            fu, fv = state
            s = (alpha * fv + tau * (self.Lap @ fu)) / tau ** 2
            return np.where(self.cls == 0, s, 0.0).astype(np.complex128)
        if self.kind == "kappa":
            fw, fz, fv = state
            div, _ = sem.interior_div_curl(self.grid, fw, fz)
            s = alpha * fv / (tau ** 2 * self.kappa) + div / tau
            return np.where(self.cls == 0, s, 0.0).astype(np.complex128)
        F1, F2, r = state
        f, g, H = self.f, self.g, self.H
        D = alpha * alpha + (tau * f) ** 2
        div, curl = sem.interior_div_curl(self.grid, F1, F2)
        s = D / (tau ** 2 * g * H * alpha) * r - (alpha * div + tau * f * curl) / (tau * g * alpha)
        out = np.where(self.cls == 0, s, 0.0).astype(np.complex128)
        xw = (self.side == 1) | (self.side == 3)
        yw = (self.side == 0) | (self.side == 2)
        out[xw] = -(alpha * F1[xw] + tau * f * F2[xw]) / (tau * g)
        out[yw] = (tau * f * F1[yw] - alpha * F2[yw]) / (tau * g)
        return out

    def post(self, alpha: complex, w: np.ndarray, state: np.ndarray) -> np.ndarray:
        """Recover all fields of (tau L - alpha)^{-1} state from the elliptic solution w."""
        tau = self.tau
        if self.kind == "wave":
            fu = state[0]
            return np.stack([(tau * w - fu) / alpha, w])
        if self.kind == "kappa":
            fw, fz, _ = state
            vx, vy = sem.gradient(self.grid, w)
            return np.stack([(tau * vx - fw) / alpha, (tau * vy - fz) / alpha, w])
        F1, F2, _ = state
        f, g = self.f, self.g
        D = alpha * alpha + (tau * f) ** 2
        hx, hy = sem.gradient(self.grid, w)
        a1 = F1 + tau * g * hx
        a2 = F2 + tau * g * hy
        U = (-alpha * a1 - tau * f * a2) / D
        V = (tau * f * a1 - alpha * a2) / D
        return np.stack([U, V, w])


class Stepper:
    """u_{n+1} = sum_m b_m (tau L - alpha_m)^{-1} u_n, factorisations cached."""

    def __init__(self, prob: Problem, alpha, b):
        self.prob = prob
        self.alpha = np.asarray(alpha, dtype=np.complex128)
        self.b = np.asarray(b, dtype=np.complex128)
        self._lu = {}

    def _solver(self, i):
        if i not in self._lu:
            self._lu[i] = spla.splu(self.prob.system(self.alpha[i]))
        return self._lu[i]

    def resolvent(self, i: int, state: np.ndarray) -> np.ndarray:
        """(tau L - alpha_i)^{-1} state (complex, all fields)."""
        a = self.alpha[i]
        w = self._solver(i).solve(self.prob.rhs(a, state))
        return self.prob.post(a, w, state)

    def step_full(self, state: np.ndarray) -> np.ndarray:
        """sum over every pole (eq. def_RM applied to tau L); complex result."""
        out = np.zeros(state.shape, dtype=np.complex128)
        for i in range(self.alpha.size):
            out += self.b[i] * self.resolvent(i, state)
        return out

    def step(self, state: np.ndarray) -> np.ndarray:
        """Real step using eq. "conjugate, matrix inverses" (Section 3.3): for a
        real state and conjugate-closed (alpha, b) only one pole of each pair is
        solved, out = Re(b_0 x_0) + 2 Re sum_{Im alpha_m > 0} b_m x_m."""
        out = np.zeros(state.shape)
        for i in range(self.alpha.size):
            im = self.alpha[i].imag
            if im < 0:
                continue
            w = 1.0 if im == 0 else 2.0
            out += w * (self.b[i] * self.resolvent(i, state)).real
        return out


def step_matrix(stepper: Stepper) -> np.ndarray:
    """Dense real matrix G of one step, column by column (G e_j): the plainest
    definition of the step's transpose is G.T.  Small grids only."""
    shape = (stepper.prob.n_fields, stepper.prob.grid.n_nodes)
    n = shape[0] * shape[1]
    G = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        G[:, j] = stepper.step(e.reshape(shape)).ravel()
    return G


def adjoint_step(stepper: Stepper, y: np.ndarray) -> np.ndarray:
    """G^T y for the real step G of Stepper.step (wave kind), factor by factor.

    With s_p = P_int (alpha_p f_v + tau A f_u) / tau^2, w_p = B_p^{-1} s_p,
    v_out = Re sum_p c_p w_p and u_out = Re sum_p (c_p tau / alpha_p) w_p - C0 f_u
    (C0 = Re sum_p c_p / alpha_p, c_p the conjugate-pair weights of Section 3.3),
    the transpose for a real seed y = (y_u, y_v) is, with the bilinear pairing,
      zeta_p = B_p^{-T} (c_p y_v + (c_p tau / alpha_p) y_u),
      u_bar = Re sum_p A^T P_int zeta_p / tau - C0 y_u,
      v_bar = Re sum_p alpha_p P_int zeta_p / tau^2.
    """
    prob = stepper.prob
    if prob.kind != "wave":
        raise NotImplementedError("adjoint_step: wave kind")
    tau = prob.tau
    yu, yv = y
    ub = np.zeros(prob.grid.n_nodes)
    vb = np.zeros(prob.grid.n_nodes)
    C0 = 0.0
    inter = (prob.cls == 0).astype(float)
    for i in range(stepper.alpha.size):
        a = stepper.alpha[i]
        if a.imag < 0:
            continue
        c = (1.0 if a.imag == 0 else 2.0) * stepper.b[i]
        z = c * yv + (c * tau / a) * yu
        zeta = stepper._solver(i).solve(z.astype(np.complex128), trans="T")
        pz = inter * zeta
        ub += (prob.Lap.T @ pz).real / tau
        vb += (a * pz).real / tau ** 2
        C0 += (c / a).real
    ub -= C0 * yu
    return np.stack([ub, vb])


def conjugate_closed(alpha, b, tol=0.0) -> bool:
    """True when the multiset {(alpha, b)} is closed under conjugation."""
    alpha = np.asarray(alpha)
    b = np.asarray(b)
    for i in range(alpha.size):
        j = np.argmin(np.abs(alpha - np.conj(alpha[i])))
        if abs(alpha[j] - np.conj(alpha[i])) > tol or abs(b[j] - np.conj(b[i])) > tol:
            return False
    return True
