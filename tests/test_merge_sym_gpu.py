"""Reflection-symmetric merge blocks (shared operators): the even/odd block apply
against the dense merge blocks of the same build (merge_dense), in FP64 and
FP32 pairs, on square, rectangular and odd-q grids (where some levels keep the
dense blocks), and against the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def state(g, seed=1000):
    x, y = g.nodes()
    c, s, a = W.draw_gaussians(seed, 3, (0.1, 0.15), (0.1, 1.0), (0.3, 0.7))
    h = W.gaussian_sum(x, y, c, s, a)
    return np.stack([0.3 * np.sin(np.pi * y) * x * (1 - x), -0.2 * np.sin(np.pi * x) * y * (1 - y), h])


@pytest.mark.parametrize("nlx,nly,p,precision", [(2, 2, 8, "fp64"), (4, 4, 10, "df32"), (4, 2, 5, "fp64"),
                                                 (2, 8, 16, "fp64"), (8, 8, 12, "df32")])
def test_symmetric_merges_match_the_dense_merges(nlx, nly, p, precision):
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(nlx, nly, p)
    kw = dict(band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True, precision=precision)
    sym = eo.Operator(g, eo.SW_WALLS, **kw)
    dense = eo.Operator(g, eo.SW_WALLS, merge_dense=True, **kw)
    u0 = state(g)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    sym.apply(a, 3)
    dense.apply(b, 3)
    e = rel(a.cpu().numpy(), b.cpu().numpy())
    print(f"{nlx}x{nly} p={p} {precision}: symmetric vs dense merges after 3 steps {e:.1e}")
    assert e <= (1e-12 if precision == "fp64" else 1e-10)


def test_symmetric_merges_match_the_oracle():
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 4, 8)
    op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True)
    u0 = state(g, 1003)
    prob = Problem(sem.Grid(4, 4, 8), "sw", op.tau, f=10.0, g=1.0, H=1.0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), Stepper(prob, op.alpha, op.b).step(u0))
    print(f"4x4 p=8 symmetric merges vs oracle: {e:.1e}")
    assert e <= 1e-10
