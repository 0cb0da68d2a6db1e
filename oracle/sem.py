"""Multidomain Chebyshev collocation of the elliptic problems (Section 2.2,
eq. Bu=f and Fig. 1), written out plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The square [x0,x1] x [y0,y1] is split into nlx x nly equal leaves, each with a
p x p tensor grid of Chebyshev-Lobatto points.  Following Section 2.2 the
elliptic operator is collocated at the (p-2)^2 interior nodes of every leaf and
continuity of the normal flux is imposed at the nodes shared by two leaves.
The four corner nodes of a leaf carry no unknown: no row below references them
(reading of the "special treatment" of corners, which the paper leaves to a
tutorial).

Public node numbering (an interface; the GPU library implements it on its own):
  interior: leaf l = b*nlx + a, local node (k, j), k, j = 1..q (q = p-2):
        id = l*q*q + (j-1)*q + (k-1)
  horizontal edge segments (y = const): line e = 0..nhl-1, leaf column a:
        id = n_int + (e*nlx + a)*q + (k-1)
  vertical edge segments (x = const): line e = 0..nvl-1, leaf row b:
        id = n_int + n_h + (b*nvl + e)*q + (j-1)
with nhl = nly + 1 and nvl = nlx + 1 lines on a walled square.  On a periodic
square (the setting of the paper's examples, Section 4) the lines y = y1 and
x = x1 are the lines y = y0 and x = x0: nhl = nly, nvl = nlx, the top edge of
leaf row nly-1 is line 0 and the right edge of leaf column nlx-1 is line 0, and
every edge node is an interface node (no domain boundary).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def cheb_points(p: int) -> np.ndarray:
    """Chebyshev-Lobatto points on [-1, 1], ascending: -cos(pi k / (p-1))."""
    k = np.arange(p)
    return -np.cos(np.pi * k / (p - 1))


def diff_matrix(x: np.ndarray) -> np.ndarray:
    """Differentiation matrix of the polynomial interpolant through nodes x.

    Barycentric form: D[i,j] = (w_j / w_i) / (x_i - x_j) for i != j with
    w_i = 1 / prod_{j != i} (x_i - x_j); the diagonal makes D @ 1 = 0.
    Exact for polynomials of degree < len(x).
    """
    n = len(x)
    w = np.array([1.0 / np.prod([x[i] - x[j] for j in range(n) if j != i]) for i in range(n)])
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return D


class Grid:
    """Leaf grid, node coordinates and the public node numbering."""

    def __init__(self, nlx: int, nly: int, p: int, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
                 periodic: bool = False):
        if p < 4:
            raise ValueError("p must be >= 4")
        self.nlx, self.nly, self.p, self.q = nlx, nly, p, p - 2
        self.x0, self.x1, self.y0, self.y1 = x0, x1, y0, y1
        self.periodic = bool(periodic)
        self.nhl = nly if self.periodic else nly + 1     # horizontal edge lines
        self.nvl = nlx if self.periodic else nlx + 1     # vertical edge lines
        self.hx = (x1 - x0) / nlx
        self.hy = (y1 - y0) / nly
        self.xi = cheb_points(p)
        D = diff_matrix(self.xi)
        self.Dx = D * (2.0 / self.hx)          # d/dx along a leaf row
        self.Dy = D * (2.0 / self.hy)          # d/dy along a leaf column
        E = diff_matrix(self.xi[1:-1])         # along one leaf edge, corners excluded
        self.Ex = E * (2.0 / self.hx)
        self.Ey = E * (2.0 / self.hy)
        q = self.q
        self.n_leaf = nlx * nly
        self.n_int = self.n_leaf * q * q
        self.n_hseg = nlx * self.nhl
        self.n_vseg = self.nvl * nly
        self.n_h = self.n_hseg * q
        self.n_v = self.n_vseg * q
        self.n_nodes = self.n_int + self.n_h + self.n_v
        self._ids = np.stack([np.stack([self._leaf_ids(a, b) for a in range(nlx)])
                              for b in range(nly)])          # [b, a, j, k]
        self.x, self.y = self._coords()

    # ------------------------------------------------------------ numbering
    def node_id(self, a: int, b: int, k: int, j: int) -> int:
        """Global id of local node (k, j) of leaf (a, b); -1 for a corner."""
        p, q = self.p, self.q
        kin = 0 < k < p - 1
        jin = 0 < j < p - 1
        if kin and jin:
            return (b * self.nlx + a) * q * q + (j - 1) * q + (k - 1)
        if kin:
            e = b if j == 0 else (b + 1) % self.nhl
            return self.n_int + (e * self.nlx + a) * q + (k - 1)
        if jin:
            e = a if k == 0 else (a + 1) % self.nvl
            return self.n_int + self.n_h + (b * self.nvl + e) * q + (j - 1)
        return -1

    def _leaf_ids(self, a, b):
        return np.array([[self.node_id(a, b, k, j) for k in range(self.p)]
                         for j in range(self.p)])

    def leaf_ids(self, a: int, b: int) -> np.ndarray:
        """p x p array of global ids of leaf (a, b), indexed [j, k]; -1 at corners."""
        return self._ids[b, a]

    def _coords(self):
        x = np.zeros(self.n_nodes)
        y = np.zeros(self.n_nodes)
        for b in range(self.nly):
            for a in range(self.nlx):
                ids = self.leaf_ids(a, b)
                X = self.x0 + (a + 0.5 * (self.xi[None, :] + 1)) * self.hx
                Y = self.y0 + (b + 0.5 * (self.xi[:, None] + 1)) * self.hy
                if self.periodic:
                    # the seam lines x = x1, y = y1 are the lines x = x0, y = y0
                    X = np.where(np.isclose(X, self.x1, rtol=0, atol=1e-14 * self.hx), self.x0, X)
                    Y = np.where(np.isclose(Y, self.y1, rtol=0, atol=1e-14 * self.hy), self.y0, Y)
                m = ids >= 0
                x[ids[m]] = np.broadcast_to(X, ids.shape)[m]
                y[ids[m]] = np.broadcast_to(Y, ids.shape)[m]
        return x, y

    def hseg_ids(self, e: int, a: int) -> np.ndarray:
        return self.n_int + (e * self.nlx + a) * self.q + np.arange(self.q)

    def vseg_ids(self, b: int, e: int) -> np.ndarray:
        return self.n_int + self.n_h + (b * self.nvl + e) * self.q + np.arange(self.q)

    def classify(self):
        """Per node: 0 interior, 1 interface, 2 domain boundary; wall side
        (0 south, 1 east, 2 north, 3 west; -1 elsewhere).  A periodic grid has
        no domain boundary: every edge node is an interface node."""
        cls = np.zeros(self.n_nodes, dtype=int)
        side = np.full(self.n_nodes, -1)
        if self.periodic:
            cls[self.n_int:] = 1
            return cls, side
        for e in range(self.nly + 1):
            for a in range(self.nlx):
                ids = self.hseg_ids(e, a)
                if e in (0, self.nly):
                    cls[ids] = 2
                    side[ids] = 0 if e == 0 else 2
                else:
                    cls[ids] = 1
        for b in range(self.nly):
            for e in range(self.nlx + 1):
                ids = self.vseg_ids(b, e)
                if e in (0, self.nlx):
                    cls[ids] = 2
                    side[ids] = 3 if e == 0 else 1
                else:
                    cls[ids] = 1
        return cls, side


# ------------------------------------------------------------------ operators

def _coo(rows, cols, vals, n):
    if not rows:                       # e.g. no interfaces on a single-leaf grid
        return sp.csr_matrix((n, n))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def divgrad_operator(g: Grid, a: np.ndarray) -> sp.csr_matrix:
    """Rows of d/dx(a du/dx) + d/dy(a du/dy) at interior nodes (zero rows elsewhere).

    Nested 1-D spectral differentiation along the node's own leaf row and
    column, with the coefficient a sampled at the nodes (Section 2.2
    collocation; a = c^2 for the wave equation, a = 1 for the Laplacian of the
    shallow-water elliptic equation).  No row references a corner node.
    """
    p = g.p
    rows, cols, vals = [], [], []
    inner = np.arange(1, p - 1)
    for b in range(g.nly):
        for a_ in range(g.nlx):
            ids = g.leaf_ids(a_, b)
            for j in inner:
                # x part on row j:  Dx[k,:] diag(a(:,j)) Dx
                arow = a[ids[j, :]]
                Mx = g.Dx[inner, :] @ (arow[:, None] * g.Dx)      # q x p
                rows.append(np.repeat(ids[j, inner], p))
                cols.append(np.tile(ids[j, :], len(inner)))
                vals.append(Mx.ravel())
            for k in inner:
                acol = a[ids[:, k]]
                My = g.Dy[inner, :] @ (acol[:, None] * g.Dy)      # q x p
                rows.append(np.repeat(ids[inner, k], p))
                cols.append(np.tile(ids[:, k], len(inner)))
                vals.append(My.ravel())
    return _coo(rows, cols, vals, g.n_nodes)


def flux_continuity_rows(g: Grid, a: np.ndarray) -> sp.csr_matrix:
    """Rows imposing continuity of the normal flux a du/dn at interface nodes.

    The outward fluxes of the two leaves sharing the node, each evaluated by
    spectral differentiation on its own leaf, sum to zero (Section 2.2).  On a
    periodic grid the seams x = x0 and y = y0 are interfaces too, between the
    last and the first leaf of each row or column.
    """
    p = g.p
    rows, cols, vals = [], [], []
    e0 = 0 if g.periodic else 1
    for b in range(g.nly):                      # vertical interfaces x = const
        for e in range(e0, g.nlx):
            L = g.leaf_ids((e - 1) % g.nlx, b)
            R = g.leaf_ids(e, b)
            for j in range(1, p - 1):
                r = L[j, p - 1]
                rows.append(np.full(2 * p, r))
                cols.append(np.concatenate([L[j, :], R[j, :]]))
                vals.append(a[r] * np.concatenate([g.Dx[p - 1, :], -g.Dx[0, :]]))
    for e in range(e0, g.nly):                  # horizontal interfaces y = const
        for a_ in range(g.nlx):
            B = g.leaf_ids(a_, (e - 1) % g.nly)
            T = g.leaf_ids(a_, e)
            for k in range(1, p - 1):
                r = B[p - 1, k]
                rows.append(np.full(2 * p, r))
                cols.append(np.concatenate([B[:, k], T[:, k]]))
                vals.append(a[r] * np.concatenate([g.Dy[p - 1, :], -g.Dy[0, :]]))
    return _coo(rows, cols, vals, g.n_nodes)


def wall_gradient_rows(g: Grid):
    """Sparse (Gx, Gy): d/dx and d/dy at domain-boundary nodes.

    Normal component: one-sided spectral derivative on the single adjacent
    leaf.  Tangential component: derivative of the interpolant through the
    p-2 non-corner nodes of that leaf edge.  Rows vanish off the boundary
    (everywhere on a periodic grid).
    """
    p = g.p
    rx, cx, vx, ry, cy, vy = [], [], [], [], [], []
    if g.periodic:
        n = g.n_nodes
        return _coo(rx, cx, vx, n), _coo(ry, cy, vy, n)
    for b in range(g.nly):
        for a_, kk in ((0, 0), (g.nlx - 1, p - 1)):
            ids = g.leaf_ids(a_, b)
            for j in range(1, p - 1):
                r = ids[j, kk]
                rx.append(np.full(p, r)); cx.append(ids[j, :]); vx.append(g.Dx[kk, :])
                ry.append(np.full(p - 2, r)); cy.append(ids[1:p - 1, kk]); vy.append(g.Ey[j - 1, :])
    for a_ in range(g.nlx):
        for b, jj in ((0, 0), (g.nly - 1, p - 1)):
            ids = g.leaf_ids(a_, b)
            for k in range(1, p - 1):
                r = ids[jj, k]
                ry.append(np.full(p, r)); cy.append(ids[:, k]); vy.append(g.Dy[jj, :])
                rx.append(np.full(p - 2, r)); cx.append(ids[jj, 1:p - 1]); vx.append(g.Ex[k - 1, :])
    n = g.n_nodes
    return _coo(rx, cx, vx, n), _coo(ry, cy, vy, n)


def gradient(g: Grid, u: np.ndarray):
    """(du/dx, du/dy) at every node.

    interior nodes: leaf spectral derivatives along the node's row / column;
    edge nodes: normal component = mean of the one-sided leaf derivatives of
    the leaves that touch the edge (one at the domain boundary, two at an
    interface, where flux continuity makes them agree); tangential component =
    derivative of the edge interpolant through its p-2 non-corner nodes.
    """
    p, q = g.p, g.q
    ux = np.zeros(g.n_nodes, dtype=u.dtype)
    uy = np.zeros(g.n_nodes, dtype=u.dtype)
    cnt_x = np.zeros(g.n_nodes)
    cnt_y = np.zeros(g.n_nodes)
    inner = np.arange(1, p - 1)
    for b in range(g.nly):
        for a_ in range(g.nlx):
            ids = g.leaf_ids(a_, b)
            U = np.zeros((p, p), dtype=u.dtype)
            m = ids >= 0
            U[m] = u[ids[m]]                       # corners stay 0 and are never used
            dX = U[inner, :] @ g.Dx.T              # rows j = 1..q, all k: d/dx
            dY = g.Dy @ U[:, inner]                # all j, columns k = 1..q: d/dy
            ii = ids[np.ix_(inner, inner)]
            ux[ii] = dX[:, inner]
            uy[ii] = dY[inner, :]
            for kk in (0, p - 1):                  # W / E edges: normal = x
                r = ids[inner, kk]
                np.add.at(ux, r, dX[:, kk]); np.add.at(cnt_x, r, 1)
            for jj in (0, p - 1):                  # S / N edges: normal = y
                r = ids[jj, inner]
                np.add.at(uy, r, dY[jj, :]); np.add.at(cnt_y, r, 1)
    e_ = cnt_x > 0
    ux[e_] /= cnt_x[e_]
    e_ = cnt_y > 0
    uy[e_] /= cnt_y[e_]
    for e in range(g.nhl):
        for a_ in range(g.nlx):
            ids = g.hseg_ids(e, a_)
            ux[ids] = g.Ex @ u[ids]
    for b in range(g.nly):
        for e in range(g.nvl):
            ids = g.vseg_ids(b, e)
            uy[ids] = g.Ey @ u[ids]
    return ux, uy


def gradient_matrices(g: Grid):
    """Sparse (Gx, Gy) with Gx @ u, Gy @ u equal to gradient(g, u): the same rules
    written as matrix rows (interior nodes: the leaf's own row / column
    differentiation; edge nodes: mean of the one-sided normal derivatives of the
    touching leaves, tangential derivative of the edge interpolant)."""
    p, n = g.p, g.n_nodes
    inner = np.arange(1, p - 1)
    rx, cx, vx, ry, cy, vy = [], [], [], [], [], []
    cnt_x = np.zeros(n)
    cnt_y = np.zeros(n)
    for b in range(g.nly):
        for a_ in range(g.nlx):
            ids = g.leaf_ids(a_, b)
            for j in inner:                                  # rows j: d/dx of interior and W/E nodes
                for k in range(p):
                    r = ids[j, k]
                    if k in (0, p - 1):
                        cnt_x[r] += 1
                    rx.append(np.full(p, r)); cx.append(ids[j, :]); vx.append(g.Dx[k, :])
            for k in inner:                                  # columns k: d/dy of interior and S/N nodes
                for j in range(p):
                    r = ids[j, k]
                    if j in (0, p - 1):
                        cnt_y[r] += 1
                    ry.append(np.full(p, r)); cy.append(ids[:, k]); vy.append(g.Dy[j, :])
    Gx = _coo(rx, cx, vx, n).tolil()
    Gy = _coo(ry, cy, vy, n).tolil()
    # interior rows were added once per leaf; edge-node normal rows once per touching leaf: mean
    sx = np.where(cnt_x > 0, 1.0 / np.maximum(cnt_x, 1), 1.0)
    sy = np.where(cnt_y > 0, 1.0 / np.maximum(cnt_y, 1), 1.0)
    Gx = sp.diags(sx) @ Gx.tocsr()
    Gy = sp.diags(sy) @ Gy.tocsr()
    Gx, Gy = Gx.tolil(), Gy.tolil()
    # tangential components on edges: rows replaced by the edge-interpolant derivative
    for e in range(g.nhl):
        for a_ in range(g.nlx):
            ids = g.hseg_ids(e, a_)
            for t, r in enumerate(ids):
                Gx.rows[r] = []
                Gx.data[r] = []
                for m, c in enumerate(ids):
                    Gx[r, c] = g.Ex[t, m]
    for b in range(g.nly):
        for e in range(g.nvl):
            ids = g.vseg_ids(b, e)
            for t, r in enumerate(ids):
                Gy.rows[r] = []
                Gy.data[r] = []
                for m, c in enumerate(ids):
                    Gy[r, c] = g.Ey[t, m]
    return Gx.tocsr(), Gy.tocsr()


def curl_of_gradient(g: Grid) -> sp.csr_matrix:
    """Interior rows of Curl(G h) = d/dx (G_y h) - d/dy (G_x h), with the interior
    derivatives of interior_div_curl applied to the recovered gradient G (zero
    rows elsewhere).  Zero in the continuum; on this discretisation nonzero at
    interior nodes next to leaf edges (tangential edge derivatives)."""
    Gx, Gy = gradient_matrices(g)
    cls, _ = g.classify()
    P = sp.diags((cls == 0).astype(float))
    return (P @ (Gx @ Gy - Gy @ Gx)).tocsr()


def interior_div_curl(g: Grid, F1: np.ndarray, F2: np.ndarray):
    """(dF1/dx + dF2/dy, dF2/dx - dF1/dy) at interior nodes (zero elsewhere),
    by leaf spectral differentiation along rows / columns."""
    f1x, f1y = gradient(g, F1)
    f2x, f2y = gradient(g, F2)
    cls, _ = g.classify()
    inside = cls == 0
    div = np.where(inside, f1x + f2y, 0.0)
    curl = np.where(inside, f2x - f1y, 0.0)
    return div, curl


def leaf_weights(g: Grid) -> np.ndarray:
    """Clenshaw-Curtis quadrature weight of every node (corners dropped), for
    discrete L2 norms and energies.  Weights of nodes shared by two leaves add."""
    p = g.p
    n = p - 1
    # Clenshaw-Curtis weights on [-1,1] for the Chebyshev-Lobatto points
    theta = np.pi * np.arange(p) / n
    w = np.zeros(p)
    v = np.ones(p - 2)
    if n % 2 == 0:
        w[0] = w[n] = 1.0 / (n * n - 1)
        for k in range(1, n // 2):
            v -= 2 * np.cos(2 * k * theta[1:-1]) / (4 * k * k - 1)
        v -= np.cos(n * theta[1:-1]) / (n * n - 1)
    else:
        w[0] = w[n] = 1.0 / (n * n)
        for k in range(1, (n - 1) // 2 + 1):
            v -= 2 * np.cos(2 * k * theta[1:-1]) / (4 * k * k - 1)
    w[1:-1] = 2 * v / n
    W2 = np.outer(w, w) * (g.hx / 2) * (g.hy / 2)
    out = np.zeros(g.n_nodes)
    for b in range(g.nly):
        for a_ in range(g.nlx):
            ids = g.leaf_ids(a_, b)
            m = ids >= 0
            np.add.at(out, ids[m], W2[m])
    return out
