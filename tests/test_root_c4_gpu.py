"""The rotation-symmetric root wall solve (square walled domain): the four
Fourier blocks against the dense wall inverse of the same build (root_dense),
forward and transposed, FP64 and FP32 pairs; and against the oracle (the
shallow-water parity tests on square grids take this path by default)."""
import numpy as np
import pytest

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def build(eo, nl, p, precision, root_dense, shared=True, consistent=False):
    g = eo.Grid(nl, nl, p)
    op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=shared,
                     precision=precision, root_dense=root_dense, sw_consistent=consistent, dense_leaves=consistent)
    return g, op


def state(g, seed=1000):
    x, y = g.nodes()
    c, s, a = W.draw_gaussians(seed, 3, (0.1, 0.15), (0.1, 1.0), (0.3, 0.7))
    h = W.gaussian_sum(x, y, c, s, a)
    return np.stack([0.3 * np.sin(np.pi * y) * x * (1 - x), -0.2 * np.sin(np.pi * x) * y * (1 - y), h])


@pytest.mark.parametrize("nl,p,precision,shared", [(2, 8, "fp64", True), (4, 10, "fp64", True),
                                                   (4, 10, "df32", True), (2, 8, "fp64", False),
                                                   (8, 12, "df32", True)])
def test_fourier_blocks_match_the_dense_root(nl, p, precision, shared):
    import paper_1402_5168_gb300 as eo
    g, c4 = build(eo, nl, p, precision, False, shared)
    _, dense = build(eo, nl, p, precision, True, shared)
    b4, bd = c4.memory()[0], dense.memory()[0]
    u0 = state(g)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    c4.apply(a, 3)
    dense.apply(b, 3)
    e = rel(a.cpu().numpy(), b.cpu().numpy())
    ya = torch.tensor(u0, device="cuda")
    yb = torch.tensor(u0, device="cuda")
    c4.apply_adjoint(ya, 2)
    dense.apply_adjoint(yb, 2)
    et = rel(ya.cpu().numpy(), yb.cpu().numpy())
    print(f"{nl}x{nl} p={p} {precision} shared={shared}: forward {e:.1e}, adjoint {et:.1e}, "
          f"operator bytes {b4 / 1e6:.1f} vs {bd / 1e6:.1f} MB")
    assert e <= 1e-11 and et <= 1e-11
    assert b4 < bd


def test_symmetric_root_matches_the_oracle_and_the_consistent_form_builds():
    import paper_1402_5168_gb300 as eo
    g, op = build(eo, 4, 8, "fp64", False)
    u0 = state(g, 1001)
    prob = Problem(sem.Grid(4, 4, 8), "sw", op.tau, f=10.0, g=1.0, H=1.0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), Stepper(prob, op.alpha, op.b).step(u0))
    print(f"4x4 p=8 symmetric root vs oracle: {e:.1e}")
    assert e <= 1e-10
    # the consistent elimination keeps the quarter-turn symmetry (the build checks it)
    g2, opc = build(eo, 2, 8, "fp64", False, consistent=True)
    probc = Problem(sem.Grid(2, 2, 8), "sw", opc.tau, f=10.0, g=1.0, H=1.0, consistent=True)
    u0 = state(g2, 1002)
    u = torch.tensor(u0, device="cuda")
    opc.apply(u, 1)
    e = rel(u.cpu().numpy(), Stepper(probc, opc.alpha, opc.b).step(u0))
    print(f"2x2 p=8 consistent, symmetric root vs oracle: {e:.1e}")
    assert e <= 1e-10
