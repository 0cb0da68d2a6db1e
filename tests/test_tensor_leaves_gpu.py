"""Leaf interior solves with the pole sum on the tensor cores (opts.tensor_leaves):
bf16 slices of the dense leaf operators [X | Y] and of the right-hand sides,
tcgen05.mma with FP32 accumulation in TMEM.

Against the FP64 oracle, column by column (tolerance TOL: the precision class of the
bf16 split, between FP32 and FP64):
* the wave equation with per-box operators (variable c, p = 16: two M tiles of the
  196 interior rows), 40 right-hand sides (a full and a ragged tile of 32 columns);
* rotating shallow water on a periodic square in the consistent elimination,
  shared dense leaf operators (every leaf a column of one product per pole);
and the same handles' FP32-pair CUDA-core path beside them.  The device status word
must stay clear (no bounded wait gave up).
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# The split keeps 41 bits of every operator entry and right-hand side (6 slices of 7
# bits), with the first three product levels exact: about 2^-41 relative per product,
# amplified by the cancellation of each step's pole sum.  Measured: 2-4e-10 (wave),
# 2.5e-9 (periodic shallow water, whose solves carry a larger cancellation).
TOL = 1e-8


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def status_ok(op):
    from paper_1402_5168_gb300 import _capi
    flag = C.c_int(-1)
    st = _capi.lib().eo_device_status(op._h, C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(flag))
    return st == 0 and flag.value == 0


def test_tensor_leaves_wave_per_box_40_rhs():
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 4, 16)
    x, y = g.nodes()
    c = W.wave_c_sincos(x, y)
    R = 40
    kw = dict(band=300.0, n_poles=21, c2=c * c, max_rhs=R, precision="df32")
    tc = eo.Operator(g, eo.WAVE_DIRICHLET, tensor_leaves=True, **kw)
    cc = eo.Operator(g, eo.WAVE_DIRICHLET, **kw)
    w = W.dataclasses.replace(W.WAVE_32X32_P16, nlx=4, nly=4)
    U0 = np.stack([np.stack(W.initial_fields(w, x, y, r)) for r in range(R)])
    a = torch.tensor(U0, device="cuda")
    b = torch.tensor(U0, device="cuda")
    tc.apply(a, 1)
    cc.apply(b, 1)
    torch.cuda.synchronize()
    assert status_ok(tc)
    got, ref = a.cpu().numpy(), b.cpu().numpy()
    st = Stepper(Problem(sem.Grid(4, 4, 16), "wave", tc.tau, c2=c * c), tc.alpha, tc.b)
    worst = 0.0
    for r in (0, 1, 17, 31, 32, 39):
        want = st.step(U0[r])
        e, e2 = rel(got[r], want), rel(ref[r], want)
        worst = max(worst, e)
        print(f"tensor leaves, wave 4x4/p16, rhs {r}: vs oracle {e:.3e} (CUDA-core FP32 pairs {e2:.3e})")
    print(f"tensor vs CUDA-core path, all 40 columns: {rel(got, ref):.3e}")
    assert worst <= TOL


def test_tensor_leaves_periodic_sw_shared():
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 4, 16, periodic=True)
    x, y = g.nodes()
    kw = dict(band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True, precision="df32", sw_consistent=True)
    tc = eo.Operator(g, eo.SW_WALLS, tensor_leaves=True, **kw)
    w = W.dataclasses.replace(W.SW_PERIODIC_16X16_P16, nlx=4, nly=4)
    s0 = np.stack(W.initial_fields(w, x, y))
    s0[0] = 0.3 * np.sin(2 * np.pi * y)
    u = torch.tensor(s0, device="cuda")
    tc.apply(u, 1)
    torch.cuda.synchronize()
    assert status_ok(tc)
    og = sem.Grid(4, 4, 16, periodic=True)
    want = Stepper(Problem(og, "sw", tc.tau, f=10.0, g=1.0, H=1.0, consistent=True), tc.alpha, tc.b).step(s0)
    e = rel(u.cpu().numpy(), want)
    print(f"tensor leaves, periodic SW 4x4/p16 shared: vs oracle {e:.3e}")
    assert e <= TOL


def test_tensor_leaves_rejected_where_not_built():
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300 import ExpopError
    g = eo.Grid(2, 2, 8)
    with pytest.raises(ExpopError, match="tensor_leaves"):
        eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, shared_ops=True, precision="df32",
                    tensor_leaves=True)   # fast-diagonal leaves are in use
    with pytest.raises(ExpopError, match="tensor_leaves"):
        x, y = g.nodes()
        eo.Operator(g, eo.WAVE_DIRICHLET, band=60.0, n_poles=21, c2=np.ones_like(x), precision="fp64",
                    tensor_leaves=True)
