"""FP32 operator storage (operators built in FP64, rounded to FP32; block
products in FP32; vectors, pole sums and pre/post maps in FP64): error against
the FP64 oracle after one and several steps, and agreement with the FP64 apply
of the same library."""
import numpy as np
import pytest

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_fp32_wave_config0_error():
    import paper_1402_5168_gb300 as eo
    w = W.WAVE_4X4_P12
    g = eo.Grid(w.nlx, w.nly, w.p)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    op32 = eo.Operator(g, eo.WAVE_DIRICHLET, band=W.BAND[w.name], n_poles=w.n_poles, c2=c * c, precision="fp32")
    op64 = eo.Operator(g, eo.WAVE_DIRICHLET, band=W.BAND[w.name], n_poles=w.n_poles, c2=c * c)
    ob32, _ = op32.memory()
    ob64, _ = op64.memory()
    assert ob32 * 2 == ob64
    prob = Problem(sem.Grid(w.nlx, w.nly, w.p), "wave", op64.tau, c2=c * c)
    st = Stepper(prob, op64.alpha, op64.b)
    u0 = np.stack(W.initial_fields(w, x, y))
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    s = u0.copy()
    errs = []
    for k in range(w.steps):
        op32.apply(a, 1)
        op64.apply(b, 1)
        s = st.step(s)
        errs.append(rel(a.cpu().numpy(), s))
    e64 = rel(b.cpu().numpy(), s)
    print(f"fp32 wave 4x4/p12: error after 1 step {errs[0]:.2e}, after {w.steps} steps {errs[-1]:.2e}; fp64 {e64:.2e}")
    assert errs[0] < 1e-5 and errs[-1] < 1e-4
    assert e64 < 1e-10


def test_fp32_sw_shared_error():
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 4, 10)
    x, y = g.nodes()
    op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True,
                     precision="fp32")
    prob = Problem(sem.Grid(4, 4, 10), "sw", op.tau, f=10.0, g=1.0, H=1.0)
    h = np.exp(-((x - 0.5) ** 2 + (y - 0.45) ** 2) / (2 * 0.12 ** 2))
    u0 = np.stack([0 * h, 0 * h, h])
    want = Stepper(prob, op.alpha, op.b).step(u0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), want)
    print(f"fp32 shallow water 4x4/p10 shared: one-step error {e:.2e}")
    assert e < 1e-5


def test_df32_wave_config0_parity():
    # FP32-pair operators: FP64-level agreement with the oracle, one step and ten
    import paper_1402_5168_gb300 as eo
    w = W.WAVE_4X4_P12
    g = eo.Grid(w.nlx, w.nly, w.p)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    op = eo.Operator(g, eo.WAVE_DIRICHLET, band=W.BAND[w.name], n_poles=w.n_poles, c2=c * c, precision="df32")
    prob = Problem(sem.Grid(w.nlx, w.nly, w.p), "wave", op.tau, c2=c * c)
    st = Stepper(prob, op.alpha, op.b)
    u0 = np.stack(W.initial_fields(w, x, y))
    a = torch.tensor(u0, device="cuda")
    s = u0.copy()
    worst = 0.0
    for k in range(w.steps):
        one = torch.tensor(s, device="cuda")
        op.apply(one, 1)
        s_next = st.step(s)
        worst = max(worst, rel(one.cpu().numpy(), s_next))
        op.apply(a, 1)
        s = s_next
    traj = rel(a.cpu().numpy(), s)
    print(f"df32 wave 4x4/p12: worst one-step {worst:.2e}, ten-step trajectory {traj:.2e}")
    assert worst <= 1e-10 and traj <= 1e-9


def test_df32_sw_shared_parity_and_adjoint_consistency():
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 4, 10)
    x, y = g.nodes()
    op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True,
                     precision="df32")
    prob = Problem(sem.Grid(4, 4, 10), "sw", op.tau, f=10.0, g=1.0, H=1.0)
    h = np.exp(-((x - 0.5) ** 2 + (y - 0.45) ** 2) / (2 * 0.12 ** 2))
    u0 = np.stack([0.1 * np.sin(np.pi * y) * x * (1 - x), 0 * h, h])
    want = Stepper(prob, op.alpha, op.b).step(u0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), want)
    print(f"df32 shallow water 4x4/p10 shared: one-step error {e:.2e}")
    assert e <= 1e-10


def test_df32_wave_adjoint_matches_fp64_adjoint():
    import paper_1402_5168_gb300 as eo
    w = W.WAVE_4X4_P12
    g = eo.Grid(4, 4, 10)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    opd = eo.Operator(g, eo.WAVE_DIRICHLET, band=250.0, n_poles=21, c2=c * c, precision="df32")
    op64 = eo.Operator(g, eo.WAVE_DIRICHLET, band=250.0, n_poles=21, c2=c * c)
    rng = np.random.default_rng(21)
    yv = rng.standard_normal((2, g.n_nodes))
    a = torch.tensor(yv, device="cuda")
    b = torch.tensor(yv, device="cuda")
    opd.apply_adjoint(a, 2)
    op64.apply_adjoint(b, 2)
    e = rel(a.cpu().numpy(), b.cpu().numpy())
    print(f"df32 adjoint vs fp64 adjoint, two steps: {e:.2e}")
    assert e <= 1e-10
