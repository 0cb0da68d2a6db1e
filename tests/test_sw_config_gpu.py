"""Shallow water on the full 16x16-leaf, p = 16 grid with tau = 20 inertial periods
(thousands of poles, shared per-level operators): parity on sampled outputs the
oracle can compute one by one (single resolvents), and a property that holds
at any size (the geostrophic steady state is left unchanged by a step)."""
import numpy as np
import pytest

import workloads as W
from oracle import rational, sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def cfg():
    import paper_1402_5168_gb300 as eo
    w = W.SW_16X16_P16
    pr = w.params
    g = eo.Grid(w.nlx, w.nly, w.p)
    op = eo.Operator(g, eo.SW_WALLS, band=W.BAND[w.name], tau=w.tau, f=pr["f"], g=pr["g"], H=pr["H"],
                     shared_ops=True)
    return w, g, op


def test_full_size_poles_meet_the_contract_near_the_band_edge(cfg):
    w, g, op = cfg
    # brute force on the band edges and beyond (the full-axis check of this many
    # poles is done by the library's fitter); conjugate closure exactly
    assert np.array_equal(op.alpha[::-1], np.conj(op.alpha))
    th = np.concatenate([np.linspace(0, 40, 2001), np.linspace(op.X - 40, op.X, 2001)])
    err = np.abs(np.exp(1j * th) - rational.R_eval(1j * th, op.alpha, op.b)).max()
    assert err <= 1e-10
    y = np.linspace(op.X, op.X + 200, 10001)
    assert np.abs(rational.R_eval(1j * y, op.alpha, op.b)).max() <= 1.0 + 1e-12


def test_full_size_sampled_resolvents(cfg):
    w, g, op = cfg
    pr = w.params
    og = sem.Grid(w.nlx, w.nly, w.p)
    prob = Problem(og, "sw", op.tau, f=pr["f"], g=pr["g"], H=pr["H"])
    st = Stepper(prob, op.alpha, op.b)
    x, y = g.nodes()
    u0 = np.stack(W.initial_fields(w, x, y))
    u = torch.tensor(u0, device="cuda")
    M = (op.alpha.size - 1) // 2
    for j in (M, M + (M // 2), 2 * M):        # real pole, mid band, outermost
        xg = torch.zeros((3, g.n_nodes), dtype=torch.complex128, device="cuda")
        op.resolvent(j, u, xg)
        want = st.resolvent(j, u0)
        e = rel(xg.cpu().numpy(), want)
        print(f"resolvent j={j} alpha={op.alpha[j]:.3f} rel {e:.3e}")
        assert e <= 1e-10


def test_full_size_geostrophic_state_is_steady(cfg):
    w, g, op = cfg
    f = w.params["f"]
    x, y = g.nodes()
    h = np.sin(np.pi * x) * np.sin(np.pi * y)
    s0 = np.stack([-(1.0 / f) * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y),
                   (1.0 / f) * np.pi * np.cos(np.pi * x) * np.sin(np.pi * y), h])
    u = torch.tensor(s0, device="cuda")
    op.apply(u, 2)
    e = rel(u.cpu().numpy(), s0)
    print(f"geostrophic state after two steps of tau = {op.tau:.4f}: rel change {e:.3e}")
    assert e <= 1e-8
