"""Symmetries of the discretisation that the library's split operators rely on,
checked on the oracle's global collocation system (Section 2.2): the quarter turn
of a square walled domain (the wall system's four Fourier blocks) and the two
reflections of a box (the even/odd merge blocks).  The oracle shares no code
with the library; these pins say the symmetries hold for the discrete problem
itself, not only for the PDE."""
import numpy as np
import pytest

from oracle import sem
from oracle.resolvent import Problem


def node_map(g, fx, fy):
    key = {(round(a, 11), round(b, 11)): i for i, (a, b) in enumerate(zip(g.x, g.y))}
    return np.array([key[(round(fx(a, b), 11), round(fy(a, b), 11))] for a, b in zip(g.x, g.y)])


def row_signs(A, pi):
    """s with A[pi r, pi c] = s_r A[r, c] for every row, or None."""
    Ad = A.toarray()
    R = Ad[np.ix_(pi, pi)]
    s = np.zeros(Ad.shape[0])
    for r in range(Ad.shape[0]):
        j = np.argmax(np.abs(Ad[r]))
        s[r] = (R[r, j] / Ad[r, j]).real
        if abs(abs(s[r]) - 1) > 1e-12 or np.abs(R[r] - s[r] * Ad[r]).max() > 1e-11 * np.abs(Ad[r]).max():
            return None
    return s


@pytest.mark.parametrize("nl,p,consistent", [(2, 8, False), (4, 6, False), (2, 8, True)])
def test_quarter_turn_maps_the_walled_square_onto_itself(nl, p, consistent):
    g = sem.Grid(nl, nl, p)
    prob = Problem(g, "sw", 0.05, f=10.0, g=1.0, H=1.0, consistent=consistent)
    pi = node_map(g, lambda x, y: 1 - y, lambda x, y: x)
    s = row_signs(prob.system(3.0 + 7.0j), pi)
    assert s is not None
    # rows keep their form alpha d_n h + tau f d_t h up to the per-side sign of the
    # written wall rows: -1 on S and W, +1 on E and N, so a row moving S->E or N->W flips
    sign = {0: -1.0, 1: 1.0, 2: -1.0, 3: 1.0}
    for r in range(g.n_nodes):
        want = sign[prob.side[r]] if prob.cls[r] == 2 else 1.0
        assert abs(s[r] - want) <= 1e-12


def test_wall_schur_complement_is_block_circulant():
    g = sem.Grid(2, 2, 8)
    prob = Problem(g, "sw", 0.05, f=10.0, g=1.0, H=1.0)
    A = prob.system(3.0 + 7.0j).toarray()
    w = [np.flatnonzero((prob.cls == 2) & (prob.side == k)) for k in range(4)]
    # counterclockwise order: S by ascending x, E ascending y, N descending x, W descending y
    ccw = [w[0][np.argsort(g.x[w[0]])], w[1][np.argsort(g.y[w[1]])],
           w[2][np.argsort(-g.x[w[2]])], w[3][np.argsort(-g.y[w[3]])]]
    walls = np.concatenate(ccw)
    o = np.flatnonzero(prob.cls != 2)
    B = A[np.ix_(walls, walls)] - A[np.ix_(walls, o)] @ np.linalg.solve(A[np.ix_(o, o)], A[np.ix_(o, walls)])
    nq = walls.size // 4
    sg = np.array([-1.0, 1.0, 1.0, -1.0])
    C = (np.repeat(sg, nq)[:, None]) * B
    blk = lambda k, l: C[k * nq:(k + 1) * nq, l * nq:(l + 1) * nq]
    for k in range(4):
        for d in range(4):
            assert np.abs(blk(k, (k + d) % 4) - blk(0, d)).max() <= 1e-12 * np.abs(C).max()


@pytest.mark.parametrize("f", [0.0, 10.0])
def test_reflections_keep_the_elliptic_rows(f):
    # the interior and interface rows (all a merge ever sees) are invariant under both
    # reflections of the domain; the wall rows are too, up to a sign, only without
    # rotation (the Coriolis term has a handedness)
    g = sem.Grid(2, 4, 8)
    prob = Problem(g, "sw", 0.05, f=f, g=1.0, H=1.0)
    A = prob.system(3.0 + 7.0j)
    inner = np.flatnonzero(prob.cls != 2)
    for fx, fy in [(lambda x, y: 1 - x, lambda x, y: y), (lambda x, y: x, lambda x, y: 1 - y)]:
        pi = node_map(g, fx, fy)
        Ad = A.toarray()
        R = Ad[np.ix_(pi, pi)]
        assert np.abs(R[inner] - Ad[inner]).max() <= 1e-11 * np.abs(Ad).max()
        assert (row_signs(A, pi) is not None) == (f == 0.0)
