"""Shallow water with the consistent elimination (the (tau f / alpha) Curl(G h)
term kept): GPU step against the oracle's consistent problem, shared and per-box
operators, and the adjoint's dot-product identity in that mode."""
import numpy as np
import pytest

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case(eo, nl, p, shared, precision="fp64"):
    g = eo.Grid(nl, nl, p)
    x, y = g.nodes()
    op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=shared,
                     sw_consistent=True, precision=precision)
    c, s, a = W.draw_gaussians(1000, 3, (0.1, 0.15), (0.1, 1.0), (0.3, 0.7))
    h = W.gaussian_sum(x, y, c, s, a)
    u0 = np.stack([0.3 * np.sin(np.pi * y) * x * (1 - x), -0.2 * np.sin(np.pi * x) * y * (1 - y), h])
    return g, op, u0


@pytest.mark.parametrize("nl,p,shared,precision", [(2, 8, True, "fp64"), (4, 10, True, "fp64"),
                                                   (2, 8, False, "fp64"), (4, 10, True, "df32")])
def test_consistent_step_matches_oracle(nl, p, shared, precision):
    import paper_1402_5168_gb300 as eo
    g, op, u0 = case(eo, nl, p, shared, precision)
    prob = Problem(sem.Grid(nl, nl, p), "sw", op.tau, f=10.0, g=1.0, H=1.0, consistent=True)
    want = Stepper(prob, op.alpha, op.b).step(u0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), want)
    # the paper's elimination gives a different step on the same grid
    plain = Stepper(Problem(sem.Grid(nl, nl, p), "sw", op.tau, f=10.0, g=1.0, H=1.0), op.alpha, op.b).step(u0)
    print(f"consistent {nl}x{nl} p{p} shared={shared} {precision}: vs oracle {e:.3e}, "
          f"difference to the plain elimination {rel(want, plain):.3e}")
    assert e <= 1e-10
    assert rel(want, plain) > 1e-6


def test_consistent_adjoint_dot_product():
    import paper_1402_5168_gb300 as eo
    g, op, u0 = case(eo, 2, 8, True)
    rng = np.random.default_rng(7)
    y = rng.standard_normal((3, g.n_nodes))
    gu = torch.tensor(u0, device="cuda")
    op.apply(gu, 2)
    gy = torch.tensor(y, device="cuda")
    op.apply_adjoint(gy, 2)
    lhs = float(np.sum(y * gu.cpu().numpy()))
    rhs = float(np.sum(gy.cpu().numpy() * u0))
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0)
