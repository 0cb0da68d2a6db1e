"""Error paths of the C ABI: every failure is a status code and a message, the
library never aborts, and a failed build leaves the device usable.

CPU (no GPU needed: the checks run on the host before any device work):
  * a non-finite or non-positive c^2 is rejected with EO_ERR_INVALID_ARG;
  * operators over opts.mem_budget_gb are rejected with EO_ERR_BUDGET, and the
    same request under a large enough budget passes that check.
GPU (failures injected on the host, EO_FAULT_INJECT; nothing faults on the device):
  * a leaf factorisation reporting a zero pivot gives EO_ERR_SINGULAR;
  * a failing build workspace allocation gives EO_ERR_OOM;
  * neither leaks device memory, and the next build on the device succeeds.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1402_5168_gb300 import _capi


def _grid(nl=2, p=8):
    L = _capi.lib()
    g = C.c_void_p()
    _capi.check(L.eo_grid_create(nl, nl, p, 0.0, 1.0, 0.0, 1.0, C.byref(g)))
    n = C.c_int64()
    _capi.check(L.eo_grid_info(g, C.byref(n), None, None))
    return g, n.value


def _build(g, kind, coeff, **kw):
    L = _capi.lib()
    o = _capi.Opts(delta=1e-10, max_rhs=1, **kw)
    h = C.c_void_p()
    cp = None if coeff is None else coeff.ctypes.data_as(C.POINTER(C.c_double))
    st = L.eo_build_operator(g, kind, cp, C.byref(o), None, C.byref(h))
    return st, L.eo_last_error().decode(), h


@pytest.mark.parametrize("bad", [np.nan, np.inf, 0.0, -1.0])
def test_bad_wave_coefficient_is_rejected(bad):
    g, n = _grid()
    c2 = np.ones(n)
    c2[n // 3] = bad
    st, msg, h = _build(g, _capi.WAVE_DIRICHLET, c2, n_poles=21, band=100.0)
    assert st == _capi.STATUS_CODES["EO_ERR_INVALID_ARG"], (st, msg)
    assert "c^2" in msg and not h.value
    _capi.lib().eo_grid_destroy(g)


def test_operator_budget_is_enforced_before_any_allocation():
    g, n = _grid(4, 10)
    st, msg, h = _build(g, _capi.SW_WALLS, None, n_poles=41, band=60.0, sw_f=10.0, sw_g=1.0, sw_H=1.0,
                        shared_ops=1, mem_budget_gb=1e-4)
    assert st == _capi.STATUS_CODES["EO_ERR_BUDGET"], (st, msg)
    assert "over the budget" in msg and not h.value
    need = float(msg.split("need ")[1].split(" GB")[0])
    assert 0 < need < 1.0
    _capi.lib().eo_grid_destroy(g)


gpu = pytest.mark.gpu


@gpu
@pytest.mark.parametrize("fault,code", [("singular", "EO_ERR_SINGULAR"), ("oom", "EO_ERR_OOM")])
def test_injected_build_failure_reports_and_recovers(monkeypatch, fault, code):
    torch = pytest.importorskip("torch")
    import paper_1402_5168_gb300 as eo
    torch.cuda.init()
    g, n = _grid(2, 8)
    kw = dict(n_poles=21, band=60.0, sw_f=10.0, sw_g=1.0, sw_H=1.0, shared_ops=1)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("EO_FAULT_INJECT", fault)
    st, msg, h = _build(g, _capi.SW_WALLS, None, **kw)
    assert st == _capi.STATUS_CODES[code], (st, msg)
    assert not h.value
    monkeypatch.delenv("EO_FAULT_INJECT")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # operators and workspace of the failed build are released (a few MB of slack
    # for the CUDA context's own bookkeeping)
    assert free1 >= free0 - (8 << 20), (free0, free1)
    st, msg, h = _build(g, _capi.SW_WALLS, None, **kw)
    assert st == 0, msg
    _capi.check(_capi.lib().eo_destroy(h))
    _capi.lib().eo_grid_destroy(g)
    # and the device still computes correctly through the public binding
    grid = eo.Grid(2, 2, 8)
    op = eo.Operator(grid, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, shared_ops=True)
    u = torch.zeros((3, grid.n_nodes), dtype=torch.float64, device="cuda")
    op.apply(u, 1)
    torch.cuda.synchronize()
    assert float(u.abs().max()) == 0.0
