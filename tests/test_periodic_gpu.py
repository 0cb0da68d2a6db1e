"""Periodic squares on the GPU (the setting of the paper's examples, Section 4):
the seam root solve, the wrapped node numbering, the pre/post maps across the
seams, against the FP64 oracle on the same periodic discretisation, and against the
Fourier-diagonalised exact solution of Section 4.1.

Cases: rotating shallow water in the consistent elimination (the stable discrete
problem; dense leaves, dense merges) in FP64 and FP32 pairs, on square and
rectangular grids and a single leaf; the elimination as written with fast-diagonal
leaves; the wave equation with per-box operators; and a 40-step run whose FP32-pair
trajectory stays within 1e-9 of the FP64 one on a bounded trajectory.
"""
import numpy as np
import pytest

import workloads as W
from oracle import reference, sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PAPER_T1 = (lambda X, Y: np.cos(6 * np.pi * X) * np.cos(4 * np.pi * Y) - 4 * np.sin(6 * np.pi * X) * np.sin(4 * np.pi * Y),
            lambda X, Y: np.cos(6 * np.pi * X) * np.cos(6 * np.pi * Y),
            lambda X, Y: np.sin(6 * np.pi * X) * np.cos(4 * np.pi * Y) - 0.2 * np.cos(4 * np.pi * X) * np.sin(2 * np.pi * Y))
BAND_T1 = float(np.sqrt(1.0 + (2 * np.pi * np.hypot(3, 3)) ** 2))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def sw_op(eo, g, n_poles, f, precision="fp64", consistent=True, band=BAND_T1, shared=True):
    return eo.Operator(g, eo.SW_WALLS, band=band, n_poles=n_poles, f=f, g=1.0, H=1.0, shared_ops=shared,
                       precision=precision, sw_consistent=consistent)


@pytest.mark.parametrize("precision", ["fp64", "df32"])
def test_periodic_sw_consistent_matches_oracle_and_fourier_exact(precision):
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 4, 16, periodic=True)
    x, y = g.nodes()
    op = sw_op(eo, g, 21, 1.0, precision)
    s0 = np.stack([fn(x, y) for fn in PAPER_T1])
    u = torch.tensor(s0, device="cuda")
    op.apply(u, 2)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    og = sem.Grid(4, 4, 16, periodic=True)
    st = Stepper(Problem(og, "sw", op.tau, f=1.0, g=1.0, H=1.0, consistent=True), op.alpha, op.b)
    want = st.step(st.step(s0))
    e = rel(got, want)
    ex = rel(got, reference.sw_fourier_exact(PAPER_T1, x, y, 2 * op.tau, 1.0))
    print(f"periodic SW 4x4/p16 consistent {precision}: two steps vs oracle {e:.3e}, vs Fourier-exact {ex:.3e}")
    assert e <= 1e-10
    assert ex <= 1e-9


@pytest.mark.parametrize("shape", [(2, 4, 10), (1, 1, 12), (4, 2, 8)])
def test_periodic_sw_consistent_shapes(shape):
    import paper_1402_5168_gb300 as eo
    nlx, nly, p = shape
    g = eo.Grid(nlx, nly, p, periodic=True)
    x, y = g.nodes()
    op = sw_op(eo, g, 21, 10.0, "fp64", band=60.0)
    rng = np.random.default_rng(nlx * 100 + nly * 10 + p)
    s0 = np.stack([np.sin(2 * np.pi * (x + rng.uniform())) * np.cos(2 * np.pi * y),
                   np.cos(2 * np.pi * x) * np.sin(4 * np.pi * (y + rng.uniform())),
                   np.cos(2 * np.pi * (x - y)) + 0.3 * np.sin(4 * np.pi * x)])
    u = torch.tensor(s0, device="cuda")
    op.apply(u, 1)
    torch.cuda.synchronize()
    og = sem.Grid(nlx, nly, p, periodic=True)
    want = Stepper(Problem(og, "sw", op.tau, f=10.0, g=1.0, H=1.0, consistent=True), op.alpha, op.b).step(s0)
    e = rel(u.cpu().numpy(), want)
    print(f"periodic SW {shape} consistent: one step vs oracle {e:.3e}")
    assert e <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "df32"])
def test_periodic_sw_fast_diagonal_leaves(precision):
    """The elimination as written (no curl term): shared operators with the
    fast-diagonal leaf solves."""
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 2, 12, periodic=True)
    x, y = g.nodes()
    op = sw_op(eo, g, 21, 1.0, precision, consistent=False)
    s0 = np.stack([fn(x, y) for fn in PAPER_T1])
    u = torch.tensor(s0, device="cuda")
    op.apply(u, 1)
    torch.cuda.synchronize()
    og = sem.Grid(4, 2, 12, periodic=True)
    want = Stepper(Problem(og, "sw", op.tau, f=1.0, g=1.0, H=1.0), op.alpha, op.b).step(s0)
    e = rel(u.cpu().numpy(), want)
    print(f"periodic SW 4x2/p12, fast-diagonal leaves, {precision}: one step vs oracle {e:.3e}")
    assert e <= 1e-10


def test_periodic_wave_per_box_operators():
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(2, 4, 10, periodic=True)
    x, y = g.nodes()
    c = W.wave_c_sincos(x, y)
    op = eo.Operator(g, eo.WAVE_DIRICHLET, band=60.0, n_poles=21, c2=c * c)
    u0 = np.stack([np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.5 * np.cos(4 * np.pi * y),
                   np.cos(2 * np.pi * (x + y))])
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    torch.cuda.synchronize()
    og = sem.Grid(2, 4, 10, periodic=True)
    want = Stepper(Problem(og, "wave", op.tau, c2=c * c), op.alpha, op.b).step(u0)
    e = rel(u.cpu().numpy(), want)
    print(f"periodic wave 2x4/p10: one step vs oracle {e:.3e}")
    assert e <= 1e-10


def test_periodic_sw_mixed_precision_after_many_steps():
    """On the stable discrete problem the FP32-pair trajectory stays within 1e-9 of
    the FP64 one after 40 steps, and the FP64 trajectory stays bounded."""
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 4, 12, periodic=True)
    x, y = g.nodes()
    w = W.SW_PERIODIC_16X16_P16
    s0 = np.stack(W.initial_fields(w, x, y))
    a = sw_op(eo, g, 61, 10.0, "df32", band=60.0)
    b = sw_op(eo, g, 61, 10.0, "fp64", band=60.0)
    ua = torch.tensor(s0, device="cuda")
    ub = torch.tensor(s0, device="cuda")
    norms = []
    for _ in range(40):
        a.apply(ua, 1)
        b.apply(ub, 1)
        norms.append(float(torch.linalg.vector_norm(ub)))
    e = float(torch.linalg.vector_norm(ua - ub) / torch.linalg.vector_norm(ub))
    growth = max(norms) / float(np.linalg.norm(s0))
    print(f"periodic SW 4x4/p12, 61 poles, 40 steps: df32 vs fp64 {e:.3e}, max norm growth {growth:.4f}")
    assert e <= 1e-9
    assert growth <= 2.0
