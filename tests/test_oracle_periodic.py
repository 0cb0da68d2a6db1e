"""The oracle on periodic squares (the setting of the paper's examples, Section 4)
against what the mathematics fixes.

* Numbering: a bijection onto the node set, the seams shared by the last and the
  first leaf of a row / column, every edge node an interface node.
* The Fourier-diagonalised exact solution of Section 4.1 (the paper's reference
  for its periodic shallow-water tests) against closed forms: a standing
  gravity wave (f = 0) and a steady geostrophic state (f != 0).
* The rational step against that exact solution for the paper's first test's
  initial fields (Section 4.1, the "first test case"), in both eliminations: the
  error is the approximant's delta plus the spectral discretisation error.
* The stability finding: with the consistent elimination the periodic step has
  spectral radius 1 (to rounding); the paper's elimination as written, and the
  walled problem in either elimination, have growing modes.
"""
import numpy as np
import pytest

from oracle import rational, reference, sem
from oracle.resolvent import Problem, Stepper, step_matrix


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nlx,nly,p", [(1, 1, 6), (2, 4, 8), (4, 4, 5)])
def test_periodic_numbering(nlx, nly, p):
    g = sem.Grid(nlx, nly, p, periodic=True)
    q = p - 2
    assert g.n_nodes == nlx * nly * (q * q + 2 * q)
    seen = np.zeros(g.n_nodes, dtype=int)
    for b in range(nly):
        for a in range(nlx):
            ids = g.leaf_ids(a, b)
            np.add.at(seen, ids[ids >= 0], 1)
    # interior nodes belong to one leaf, every edge node to exactly two
    assert np.all(seen[:g.n_int] == 1) and np.all(seen[g.n_int:] == 2)
    # the right edge of the last column is the left edge of the first
    for b in range(nly):
        assert np.array_equal(g.leaf_ids(nlx - 1, b)[1:-1, p - 1], g.leaf_ids(0, b)[1:-1, 0])
    for a in range(nlx):
        assert np.array_equal(g.leaf_ids(a, nly - 1)[p - 1, 1:-1], g.leaf_ids(a, 0)[0, 1:-1])
    cls, side = g.classify()
    assert np.all(cls[g.n_int:] == 1) and np.all(side == -1)
    assert g.x.min() >= 0 and g.x.max() < 1 and g.y.min() >= 0 and g.y.max() < 1


def test_fourier_reference_standing_gravity_wave():
    # f = 0: h = cos(kx) cos(wt), u = (w / (H k)) sin(kx) sin(wt), w^2 = g H k^2
    g_, H, k = 2.0, 0.5, 2 * np.pi * 3
    w = np.sqrt(g_ * H) * k
    x = np.linspace(0, 1, 37)[:-1]
    y = 0.3 + 0 * x
    t = 0.37
    got = reference.sw_fourier_exact([lambda X, Y: 0 * X, lambda X, Y: 0 * X, lambda X, Y: np.cos(k * X)],
                                     x, y, t, 0.0, g_, H, n=16)
    assert np.allclose(got[2], np.cos(k * x) * np.cos(w * t), atol=1e-13)
    assert np.allclose(got[0], w / (H * k) * np.sin(k * x) * np.sin(w * t), atol=1e-13)
    assert np.allclose(got[1], 0, atol=1e-13)


def test_fourier_reference_geostrophic_state_is_steady():
    f, g_ = 3.0, 1.5
    hh = lambda X, Y: np.sin(2 * np.pi * X) * np.cos(4 * np.pi * Y)
    u = lambda X, Y: -(g_ / f) * (-4 * np.pi) * np.sin(2 * np.pi * X) * np.sin(4 * np.pi * Y)
    v = lambda X, Y: (g_ / f) * 2 * np.pi * np.cos(2 * np.pi * X) * np.cos(4 * np.pi * Y)
    x = np.random.default_rng(3).uniform(0, 1, 50)
    y = np.random.default_rng(4).uniform(0, 1, 50)
    got = reference.sw_fourier_exact([u, v, hh], x, y, 2.7, f, g_, 1.0, n=16)
    want = np.stack([u(x, y), v(x, y), hh(x, y)])
    assert np.abs(got - want).max() <= 1e-12


# the paper's first periodic shallow-water test (Section 4.1): its eta is taken as h
PAPER_T1 = (lambda X, Y: np.cos(6 * np.pi * X) * np.cos(4 * np.pi * Y) - 4 * np.sin(6 * np.pi * X) * np.sin(4 * np.pi * Y),
            lambda X, Y: np.cos(6 * np.pi * X) * np.cos(6 * np.pi * Y),
            lambda X, Y: np.sin(6 * np.pi * X) * np.cos(4 * np.pi * Y) - 0.2 * np.cos(4 * np.pi * X) * np.sin(2 * np.pi * Y))


@pytest.fixture(scope="module")
def fit21():
    return rational.fit(21)


@pytest.mark.parametrize("consistent", [False, True])
def test_periodic_step_matches_the_fourier_exact_solution(consistent, fit21):
    g = sem.Grid(4, 4, 16, periodic=True)
    st0 = np.stack([fn(g.x, g.y) for fn in PAPER_T1])
    alpha, b, X = fit21
    tau = X / np.sqrt(1.0 + (2 * np.pi * np.hypot(3, 3)) ** 2)   # band: the data's largest frequency
    prob = Problem(g, "sw", tau, f=1.0, g=1.0, H=1.0, consistent=consistent)
    st = Stepper(prob, alpha, b)
    got = st.step(st.step(st0))
    want = reference.sw_fourier_exact(PAPER_T1, g.x, g.y, 2 * tau, 1.0)
    e = rel(got, want)
    print(f"periodic SW 4x4/p16, 21 poles, consistent={consistent}: two steps, rel L2 vs the Fourier-exact "
          f"solution {e:.3e}")
    assert e <= 1e-9


_FIT = {}


def _rho(periodic, consistent, f=10.0):
    g = sem.Grid(2, 2, 8, periodic=periodic)
    if not _FIT:
        _FIT["21"] = rational.fit(21)
    alpha, b, _ = _FIT["21"]
    prob = Problem(g, "sw", 0.05, f=f, g=1.0, H=1.0, consistent=consistent)
    return np.abs(np.linalg.eigvals(step_matrix(Stepper(prob, alpha, b)))).max()


def test_periodic_consistent_step_has_unit_spectral_radius():
    assert _rho(True, True) <= 1.0 + 1e-7


def test_growing_modes_of_the_other_discrete_problems():
    """Documented property (a finding, not a target): the paper's elimination as
    written on a periodic square, and walls in either elimination, give steps with
    spectral radius above one at f = 10."""
    assert _rho(True, False) >= 1.0 + 1e-3
    assert _rho(False, True) >= 1.0 + 1e-3
    assert _rho(False, False) >= 1.0 + 1e-3
    # without rotation every one of them is stable
    assert _rho(False, False, f=0.0) <= 1.0 + 1e-7


def test_periodic_consistent_resolvent_identity():
    """With the consistent elimination the per-pole solves are resolvents of one
    discrete operator: R(a) - R(b) = (a - b) R(a) R(b), R(a) = (tau L - a)^{-1}."""
    g = sem.Grid(2, 2, 8, periodic=True)
    prob = Problem(g, "sw", 0.3, f=10.0, g=1.0, H=1.0, consistent=True)
    al = np.array([2.0 + 1.0j, 3.0 - 2.0j])
    st = Stepper(prob, al, np.ones(2))
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3, g.n_nodes))
    ra = st.resolvent(0, u)
    rb = st.resolvent(1, u)
    rab = st.resolvent(0, st.resolvent(1, u))
    assert rel(ra - rb, (al[0] - al[1]) * rab) <= 1e-12
