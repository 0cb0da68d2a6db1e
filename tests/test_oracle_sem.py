"""Pins of oracle.sem (Section 2.2): spectral differentiation, numbering and
quadrature against closed forms."""
import pytest
import numpy as np

from oracle import sem


def test_diff_matrix_exact_on_polynomials():
    for p in (6, 12, 16):
        x = sem.cheb_points(p)
        D = sem.diff_matrix(x)
        for d in range(p):
            want = d * x ** (d - 1) if d > 0 else 0 * x
            assert np.abs(D @ x ** d - want).max() < 1e-9 * max(1, d) ** 2
        assert x[0] == -1.0 and abs(x[-1] - 1.0) < 1e-15 and np.all(np.diff(x) > 0)


def test_numbering_is_a_bijection_and_coordinates_match_leaf_grid():
    g = sem.Grid(4, 2, 7)
    seen = np.zeros(g.n_nodes, int)
    for b in range(g.nly):
        for a in range(g.nlx):
            ids = g.leaf_ids(a, b)
            assert ids[0, 0] == ids[0, -1] == ids[-1, 0] == ids[-1, -1] == -1
            assert np.all(ids[1:-1, 1:-1] < g.n_int)
            seen[ids[1:-1, 1:-1].ravel()] += 1
    assert np.all(seen[:g.n_int] == 1)
    assert g.n_nodes == 4 * 2 * 25 + 4 * 3 * 5 + 5 * 2 * 5
    # an edge node shared by two leaves has the same coordinates seen from both
    L = g.leaf_ids(0, 0)
    R = g.leaf_ids(1, 0)
    assert np.array_equal(L[1:-1, -1], R[1:-1, 0])
    assert np.allclose(g.x[L[1:-1, -1]], 0.25)
    assert np.allclose(g.y[L[1:-1, -1]], 0.5 * (sem.cheb_points(7)[1:-1] + 1) * 0.5)


def test_divgrad_on_polynomial_is_exact():
    # d/dx(a u_x) + d/dy(a u_y) with a = 1 + x + y, u = x^3 y^2 (degree < p per
    # leaf direction): closed form 3x^2y^2(...) written out below.
    g = sem.Grid(2, 2, 9)
    x, y = g.x, g.y
    a = 1 + x + y
    u = x ** 3 * y ** 2
    ux, uy = 3 * x ** 2 * y ** 2, 2 * x ** 3 * y
    want = a * (6 * x * y ** 2 + 2 * x ** 3) + ux + uy
    got = sem.divgrad_operator(g, a) @ u
    cls, _ = g.classify()
    assert np.abs((got - want)[cls == 0]).max() < 1e-9


def test_gradient_and_div_curl_exact_on_polynomials():
    g = sem.Grid(2, 3, 8)
    x, y = g.x, g.y
    u = x ** 2 * y - 3 * y ** 3
    ux, uy = sem.gradient(g, u)
    assert np.abs(ux - 2 * x * y).max() < 1e-10
    assert np.abs(uy - (x ** 2 - 9 * y ** 2)).max() < 1e-10
    F1, F2 = x * y ** 2, x ** 3 + y
    div, curl = sem.interior_div_curl(g, F1, F2)
    cls, _ = g.classify()
    m = cls == 0
    assert np.abs(div[m] - (y ** 2 + 1)[m]).max() < 1e-10
    assert np.abs(curl[m] - (3 * x ** 2 - 2 * x * y)[m]).max() < 1e-10


def test_flux_rows_vanish_on_smooth_functions():
    g = sem.Grid(3, 2, 8)
    a = 2 + np.sin(g.x)
    u = np.cos(g.x) * g.y ** 2
    r = sem.flux_continuity_rows(g, a) @ u
    assert np.abs(r).max() < 1e-9


def test_quadrature_weights():
    g = sem.Grid(2, 2, 10)
    w = sem.leaf_weights(g)
    # x(1-x)(2x-1)^2 y(1-y) vanishes at every leaf corner of the 2 x 2 grid
    # (x in {0, 1/2, 1} there), so dropping corners costs nothing; its integral
    # over the unit square is (1/30)(1/6).
    f = g.x * (1 - g.x) * (2 * g.x - 1) ** 2 * g.y * (1 - g.y)
    assert abs(w @ f - 1.0 / 180.0) < 1e-15
    assert abs(w.sum() - 1.0) < 0.02


@pytest.mark.parametrize("nl,p", [(1, 6), (2, 7), (2, 8)])
def test_gradient_matrices_equal_the_procedural_gradient(nl, p):
    g = sem.Grid(nl, nl, p)
    Gx, Gy = sem.gradient_matrices(g)
    u = np.random.default_rng(nl * 10 + p).standard_normal(g.n_nodes)
    hx, hy = sem.gradient(g, u)
    assert np.abs(Gx @ u - hx).max() <= 1e-12 * np.abs(hx).max()
    assert np.abs(Gy @ u - hy).max() <= 1e-12 * np.abs(hy).max()
    # Curl(G h) equals interior_div_curl of the recovered gradient and vanishes on
    # polynomials of the leaf degree that the edge interpolant reproduces
    c = sem.interior_div_curl(g, hx, hy)[1]
    assert np.abs(sem.curl_of_gradient(g) @ u - c).max() <= 1e-12 * np.abs(c).max()
    poly = g.x ** 2 * g.y + 0.5 * g.y ** 3 - g.x
    assert np.abs(sem.curl_of_gradient(g) @ poly).max() <= 1e-9
