"""eo_apply_resolvent_noalloc: the resolvent entry point for callers that cannot
allocate device memory when they call (graph-capture code, allocator-free host
threads, hosts that own the whole GPU through their own pool).  It must give
what eo_apply_resolvent gives, on two calls in a row, through the C ABI.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind", ["wave", "sw"])
def test_noalloc_resolvent_matches_allocating_entry_point(kind):
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300 import _capi
    L = _capi.lib()
    g = eo.Grid(4, 4, 10)
    x, y = g.nodes()
    if kind == "wave":
        c = W.wave_c(W.WAVE_4X4_P12, x, y)
        op = eo.Operator(g, eo.WAVE_DIRICHLET, band=250.0, n_poles=21, c2=c * c)
        u0 = np.stack(W.initial_fields(W.WAVE_4X4_P12, x, y))
    else:
        op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0)
        h = np.exp(-((x - 0.5) ** 2 + (y - 0.4) ** 2) / (2 * 0.1 ** 2))
        u0 = np.stack([0.1 * np.sin(np.pi * y), 0 * h, h])
    u = torch.tensor(u0, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    M = (op.alpha.size - 1) // 2
    for j in (M + 2, 2 * M):          # two calls in a row, different poles
        want = torch.zeros((op.fields, g.n_nodes), dtype=torch.complex128, device="cuda")
        got = torch.zeros_like(want)
        _capi.check(L.eo_apply_resolvent(op._h, j, C.c_void_p(u.data_ptr()), C.c_void_p(want.data_ptr()),
                                         stream))
        _capi.check(L.eo_apply_resolvent_noalloc(op._h, j, C.c_void_p(u.data_ptr()),
                                                 C.c_void_p(got.data_ptr()), stream))
        torch.cuda.synchronize()
        e = rel(got.cpu().numpy(), want.cpu().numpy())
        assert e <= 1e-10, (j, e)
