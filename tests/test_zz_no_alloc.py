"""eo_apply_resolvent_noalloc: the resolvent entry point for callers that cannot
allocate device memory when they call (host threads that must stay off the device
allocator, programs that give all of the GPU's memory to their own pool).  Through
the C ABI, on two calls in a row, it must give what eo_apply_resolvent gives, and
it must not allocate: the free device memory and the high watermark of the
device's stream-ordered memory pool (the pool cudaMallocAsync draws from) do not
move across the two calls.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# CUmemPool_attribute values of the CUDA driver API
_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class _Pool:
    """The current device's default memory pool through the driver API."""

    def __init__(self):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), C.c_int(torch.cuda.current_device())) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, C.c_int(attr), C.byref(v)) == 0
        return v.value

    def reset_high(self):
        v = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, C.c_int(_USED_MEM_HIGH), C.byref(v)) == 0


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
    poles = (M + 2, 2 * M)            # two calls in a row, different poles
    want = [torch.zeros((op.fields, g.n_nodes), dtype=torch.complex128, device="cuda") for _ in poles]
    got = [torch.zeros_like(w) for w in want]
    for j, w in zip(poles, want):
        _capi.check(L.eo_apply_resolvent(op._h, j, C.c_void_p(u.data_ptr()), C.c_void_p(w.data_ptr()), stream))
    # the first call on a device looks the scratch array up; then nothing may allocate
    scratch = torch.zeros_like(want[0])
    _capi.check(L.eo_apply_resolvent_noalloc(op._h, poles[0], C.c_void_p(u.data_ptr()),
                                             C.c_void_p(scratch.data_ptr()), stream))
    torch.cuda.synchronize()
    pool = _Pool()
    pool.reset_high()
    used0 = pool.get(_USED_MEM_CURRENT)
    free0, _ = torch.cuda.mem_get_info()
    for j, gt in zip(poles, got):
        _capi.check(L.eo_apply_resolvent_noalloc(op._h, j, C.c_void_p(u.data_ptr()),
                                                 C.c_void_p(gt.data_ptr()), stream))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    high = pool.get(_USED_MEM_HIGH)
    assert free1 == free0, ("device memory changed across the calls", free0, free1)
    assert high <= used0, ("the stream-ordered pool was drawn on", used0, high)
    for j, gt, w in zip(poles, got, want):
        e = rel(gt.cpu().numpy(), w.cpu().numpy())
        assert e <= 1e-10, (j, e)
