"""GB300 engine for repeated application of the rational time-evolution operator
exp(tau L) ~ sum_m b_m (tau L - alpha_m)^{-1} (Haut, Babb, Martinsson, Wingate).

Thin Python binding over the C ABI in ``include/expop.h``: it marshals
arguments (device pointers of torch tensors, host numpy arrays, the CUDA
stream) and does no arithmetic of its own.  Every step of the build and apply
phases runs in the compiled library ``_build/libexpop.so``; if the library is
missing the calls raise.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _capi
from ._capi import SW_WALLS, WAVE_DIRICHLET, WAVE_KAPPA, ExpopError, Opts, check

__all__ = ["Grid", "Operator", "Batch", "fit", "fit_gauss", "leaf_basis", "WAVE_DIRICHLET", "SW_WALLS", "ExpopError"]


def fit(n_poles: int = 0, X: float = 0.0, delta: float = 1e-10, cap: int = 20001):
    """Rational approximant (alpha, b, X) of e^{ix} on [-X, X]; host only."""
    a = np.zeros(2 * cap)
    b = np.zeros(2 * cap)
    n, Xo = C.c_int(), C.c_double()
    dp = C.POINTER(C.c_double)
    check(_capi.lib().eo_fit(n_poles, X, delta, cap, a.ctypes.data_as(dp), b.ctypes.data_as(dp), C.byref(n),
                             C.byref(Xo)))
    k = n.value
    return a[0:2 * k:2] + 1j * a[1:2 * k:2], b[0:2 * k:2] + 1j * b[1:2 * k:2], Xo.value


def fit_gauss(X: float, h: float = 0.18, delta: float = 1e-10):
    """The paper's Gaussian-sum approximant of e^{ix} on [-X, X] (two pole lines);
    returns (alpha, b, M).  Host only."""
    n, M = C.c_int(), C.c_int()
    dp = C.POINTER(C.c_double)
    L = _capi.lib()
    L.eo_fit_gauss(X, h, delta, 0, None, None, C.byref(n), C.byref(M))   # size query
    if n.value <= 0:
        check(L.eo_fit_gauss(X, h, delta, 0, None, None, C.byref(n), C.byref(M)))
    a = np.zeros(2 * n.value)
    b = np.zeros(2 * n.value)
    check(L.eo_fit_gauss(X, h, delta, n.value, a.ctypes.data_as(dp), b.ctypes.data_as(dp), C.byref(n),
                         C.byref(M)))
    return a[0::2] + 1j * a[1::2], b[0::2] + 1j * b[1::2], M.value


def leaf_basis(p: int, length: float = 2.0, a: float = 1.0):
    """Separable eigenbasis of a constant-coefficient leaf (host only): returns
    (lam, V, Vinv) with a (D D)_ii = V diag(lam) Vinv on p Chebyshev-Lobatto
    points of an interval of the given length (q = p - 2 interior points)."""
    q = p - 2
    lam = np.zeros(q)
    V = np.zeros((q, q))
    Vi = np.zeros((q, q))
    dp = C.POINTER(C.c_double)
    check(_capi.lib().eo_leaf_basis(p, length, a, lam.ctypes.data_as(dp), V.ctypes.data_as(dp),
                                    Vi.ctypes.data_as(dp)))
    return lam, V, Vi


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class Grid:
    """nlx x nly leaves of p x p Chebyshev nodes on [x0,x1] x [y0,y1]; periodic=True
    identifies x1 with x0 and y1 with y0 (eo_grid_create_periodic)."""

    def __init__(self, nlx, nly, p, x0=0.0, x1=1.0, y0=0.0, y1=1.0, periodic=False):
        L = _capi.lib()
        self._h = C.c_void_p()
        create = L.eo_grid_create_periodic if periodic else L.eo_grid_create
        check(create(nlx, nly, p, x0, x1, y0, y1, C.byref(self._h)))
        self.periodic = bool(periodic)
        n, ni, ne = C.c_int64(), C.c_int64(), C.c_int64()
        check(L.eo_grid_info(self._h, C.byref(n), C.byref(ni), C.byref(ne)))
        self.nlx, self.nly, self.p = nlx, nly, p
        self.n_nodes, self.n_interior, self.n_edge = n.value, ni.value, ne.value

    def nodes(self):
        x = np.zeros(self.n_nodes)
        y = np.zeros(self.n_nodes)
        check(_capi.lib().eo_grid_nodes(self._h, x.ctypes.data_as(C.POINTER(C.c_double)),
                                        y.ctypes.data_as(C.POINTER(C.c_double))))
        return x, y

    def __del__(self):
        if getattr(self, "_h", None) and _capi._lib is not None:
            _capi._lib.eo_grid_destroy(self._h)
            self._h = None


class Operator:
    """Built operator R(tau L) = sum_m b_m (tau L - alpha_m)^{-1} on one GPU."""

    def __init__(self, grid: Grid, kind: int, band: float, n_poles: int = 0, tau: float = 0.0,
                 c2=None, f=0.0, g=1.0, H=1.0, delta=1e-10, shared_ops=False, max_rhs=1,
                 mem_budget_gb=0.0, precision="fp64", fp64_top_levels=0, use_graphs=True, dense_leaves=False,
                 autotune=True, sw_consistent=False, fitter="line", gauss_h=0.0, root_dense=False,
                 merge_dense=False, tensor_leaves=False, merge_fuse=0, stream=None):
        L = _capi.lib()
        prec = {"fp64": 0, "fp32": 1, "df32": 2}[precision]
        fit_kind = {"line": 0, "gauss": 1}[fitter]
        o = Opts(n_poles=n_poles, band=band, tau=tau, delta=delta, sw_f=f, sw_g=g, sw_H=H, precision=prec,
                 shared_ops=int(shared_ops), max_rhs=max_rhs, mem_budget_gb=mem_budget_gb,
                 fp64_top_levels=fp64_top_levels, use_graphs=int(use_graphs), dense_leaves=int(dense_leaves),
                 autotune=int(autotune), sw_consistent=int(sw_consistent), fitter=fit_kind,
                 gauss_h=gauss_h, root_dense=int(root_dense), merge_dense=int(merge_dense),
                 tensor_leaves=int(tensor_leaves), merge_fuse=int(merge_fuse))
        coeff = None
        if c2 is not None:
            self._c2 = np.ascontiguousarray(c2, dtype=np.float64)
            coeff = self._c2.ctypes.data_as(C.POINTER(C.c_double))
        self._h = C.c_void_p()
        self.grid = grid
        self.kind = kind
        self.fields = 2 if kind == WAVE_DIRICHLET else 3
        self.max_rhs = max_rhs
        check(L.eo_build_operator(grid._h, kind, coeff, C.byref(o), _stream_ptr(stream), C.byref(self._h)))
        n, tau_, X = C.c_int(), C.c_double(), C.c_double()
        check(L.eo_get_poles(self._h, None, None, C.byref(n), C.byref(tau_), C.byref(X)))
        a = np.zeros(2 * n.value)
        b = np.zeros(2 * n.value)
        dp = C.POINTER(C.c_double)
        check(L.eo_get_poles(self._h, a.ctypes.data_as(dp), b.ctypes.data_as(dp), C.byref(n), None, None))
        self.alpha = a[0::2] + 1j * a[1::2]
        self.b = b[0::2] + 1j * b[1::2]
        self.tau, self.X = tau_.value, X.value

    def memory(self):
        ob, wb = C.c_int64(), C.c_int64()
        check(_capi.lib().eo_memory(self._h, C.byref(ob), C.byref(wb)))
        return ob.value, wb.value

    def apply(self, u, n_steps=1, stream=None):
        """u <- R(tau L)^n_steps u in place; u: CUDA float64 tensor [n_rhs, fields, n_nodes]
        (or [fields, n_nodes] for one state)."""
        if not (u.is_cuda and u.dtype.is_floating_point and u.element_size() == 8 and u.is_contiguous()):
            raise ValueError("u must be a contiguous CUDA float64 tensor")
        n_rhs = 1 if u.dim() == 2 else u.shape[0]
        if u.shape[-2:] != (self.fields, self.grid.n_nodes):
            raise ValueError(f"state shape must end with ({self.fields}, {self.grid.n_nodes})")
        check(_capi.lib().eo_apply(self._h, C.c_void_p(u.data_ptr()), n_rhs, n_steps, _stream_ptr(stream)))
        return u

    def apply_adjoint(self, y, n_steps=1, stream=None):
        """y <- (G^T)^n_steps y in place (G = one apply step); same layout as apply."""
        if not (y.is_cuda and y.element_size() == 8 and y.is_contiguous()):
            raise ValueError("y must be a contiguous CUDA float64 tensor")
        n_rhs = 1 if y.dim() == 2 else y.shape[0]
        check(_capi.lib().eo_apply_adjoint(self._h, C.c_void_p(y.data_ptr()), n_rhs, n_steps, _stream_ptr(stream)))
        return y

    def apply_host(self, u: np.ndarray, n_steps=1, stream=None):
        """Same as apply for a host float64 array (copies in and out inside the call)."""
        if u.dtype != np.float64 or not u.flags["C_CONTIGUOUS"]:
            raise ValueError("u must be a C-contiguous float64 array")
        n_rhs = 1 if u.ndim == 2 else u.shape[0]
        check(_capi.lib().eo_apply_host(self._h, u.ctypes.data_as(C.POINTER(C.c_double)), n_rhs, n_steps,
                                        _stream_ptr(stream)))
        return u

    def resolvent(self, j, u, x, stream=None):
        """x <- (tau L - alpha_j)^{-1} u for pole index j (Im alpha_j >= 0); u float64
        [fields, n_nodes], x complex128 [fields, n_nodes], both CUDA tensors."""
        check(_capi.lib().eo_apply_resolvent(self._h, j, C.c_void_p(u.data_ptr()), C.c_void_p(x.data_ptr()),
                                             _stream_ptr(stream)))
        return x

    def fit_function(self, kind: str = "exp", c: float = 1.0):
        """Residues (numpy complex, eo_get_poles order) of exp(c z) ("exp"), phi1(z)
        ("phi1"), phi2(z) ("phi2") or, for fitter="gauss", the partition-of-unity filter keeping a
        fraction c of the Gaussians ("filter") on this operator's poles, and the
        band error."""
        n = self.alpha.size
        b = np.zeros(2 * n)
        err = C.c_double()
        check(_capi.lib().eo_fit_function(self._h, {"exp": 0, "phi1": 1, "filter": 2, "phi2": 3}[kind], c,
                                          b.ctypes.data_as(C.POINTER(C.c_double)), C.byref(err)))
        return b[0::2] + 1j * b[1::2], err.value

    def apply_functions(self, b_sets, u, out, stream=None):
        """out[k] <- f_k(tau L) u for residue sets b_sets[k] on these poles (one
        shared sweep); u: CUDA float64 [fields, n_nodes]; out: [n_out, fields, n_nodes]."""
        bs = np.ascontiguousarray(np.stack([np.stack([np.real(b), np.imag(b)], axis=1).ravel()
                                            for b in b_sets]))
        if out.shape[0] != len(b_sets) or not out.is_contiguous() or not u.is_contiguous():
            raise ValueError("out must be contiguous [n_out, fields, n_nodes]")
        check(_capi.lib().eo_apply_functions(self._h, len(b_sets), bs.ctypes.data_as(C.POINTER(C.c_double)),
                                             C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()),
                                             _stream_ptr(stream)))
        return out

    def apply_filtered(self, u, n_steps=1, keep: float = 0.9, stream=None):
        """u <- (S(tau L) R(tau L))^n_steps u for one state [fields, n_nodes]: each step
        applies the approximant, then the filter S (residues fit_function("filter",
        keep)) on the same poles (Section 3.3).  Two sweeps per step."""
        import torch
        if not hasattr(self, "_filter") or self._filter[0] != keep:
            self._filter = (keep, self.fit_function("filter", keep)[0])
        out = torch.empty((1,) + tuple(u.shape), dtype=u.dtype, device=u.device)
        for _ in range(n_steps):
            self.apply(u, 1, stream)
            self.apply_functions([self._filter[1]], u, out, stream)
            u.copy_(out[0])
        return u

    def apply_laplacian_filter(self, s, u, stream=None):
        """u <- S(k0 Delta) u field by field, in place (eo_apply_laplacian_filter): s the
        filter's residues on this operator's poles; this operator a shallow-water one
        with f = 0 (k0 = tau^2 g H); u: CUDA float64 [n_rhs, fields, n_nodes] or
        [fields, n_nodes] of any state on this grid."""
        if not (u.is_cuda and u.element_size() == 8 and u.is_contiguous()) or u.shape[-1] != self.grid.n_nodes:
            raise ValueError("u must be a contiguous CUDA float64 tensor [..., fields, n_nodes]")
        n_fields = u.shape[-2]
        n_rhs = 1 if u.dim() == 2 else u.shape[0]
        ss = np.ascontiguousarray(np.stack([np.real(s), np.imag(s)], axis=1).ravel())
        check(_capi.lib().eo_apply_laplacian_filter(self._h, ss.ctypes.data_as(C.POINTER(C.c_double)),
                                                    C.c_void_p(u.data_ptr()), n_fields, n_rhs, _stream_ptr(stream)))
        return u

    def fused_levels(self, n_rhs: int = 1) -> int:
        """Merge levels 1 .. n run in one launch per sweep for n_rhs right-hand sides."""
        n = C.c_int(-1)
        check(_capi.lib().eo_fused_levels(self._h, n_rhs, C.byref(n)))
        return n.value

    def set_timing(self, on: bool):
        check(_capi.lib().eo_set_timing(self._h, int(on)))

    def timing(self):
        """{kernel class: (launches, device ms)} since the previous call."""
        n = C.c_int(16)
        names = (C.c_char_p * 16)()
        launches = (C.c_int64 * 16)()
        ms = (C.c_double * 16)()
        check(_capi.lib().eo_get_timing(self._h, C.byref(n), names, launches, ms))
        return {names[i].decode(): (launches[i], ms[i]) for i in range(n.value)}

    def close(self):
        if getattr(self, "_h", None) and _capi._lib is not None:
            _capi._lib.eo_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class LaplacianFilter:
    """S(k0 Delta) of Section 3.3 on a grid: the rational partition of unity of the
    Gaussian-sum construction (M Gaussians of width h fitted on |theta| <= X; the window
    keeps M0 = floor(keep M) of them) applied to the Laplacian.  It runs through a
    shallow-water operator with f = 0, g = H = 1 and tau = sqrt(k0), whose per-pole
    solve is (k0 Delta - alpha^2) w = alpha r: a mode of wavenumber |k| is multiplied by
    about chi(sqrt(k0) |k| / 2 pi), flat (to 1e-10) for sqrt(k0) |k| / 2 pi below about
    (M0 - 10) h and zero beyond (M0 + 10) h."""

    def __init__(self, grid: Grid, k0: float, X: float = 30.0, keep: float = 0.9, h: float = 0.18,
                 precision: str = "fp64", max_rhs: int = 1):
        if not k0 > 0:
            raise ValueError("k0 must be positive")
        tau = float(np.sqrt(k0))
        self.k0, self.h = float(k0), float(h)
        self.op = Operator(grid, SW_WALLS, band=X / tau, tau=tau, f=0.0, g=1.0, H=1.0, shared_ops=True,
                           fitter="gauss", gauss_h=h, precision=precision, max_rhs=max_rhs)
        self.s, self.err = self.op.fit_function("filter", keep)
        self.M = (self.op.alpha.size // 2 - 1) // 2 - 11
        self.M0 = int(np.floor(keep * self.M))

    @staticmethod
    def k0_keeping(k_over_2pi: float, M0: int, h: float = 0.18) -> float:
        """k0 that keeps the window flat up to |k| / 2 pi = k_over_2pi (edge margin 10 h)."""
        return float(((M0 - 10) * h / k_over_2pi) ** 2)

    def apply(self, u, stream=None):
        """u <- S(k0 Delta) u, every field of every right-hand side, in place."""
        return self.op.apply_laplacian_filter(self.s, u, stream)


class Batch:
    """Independent instances (operators with their own device states) advanced
    together: one step pair of every instance is recorded as parallel branches of
    one CUDA graph and replayed (eo_batch_create / eo_batch_apply)."""

    def __init__(self, ops, states):
        if len(ops) != len(states) or not ops:
            raise ValueError("need one state per operator")
        n = len(ops)
        for op, u in zip(ops, states):
            if not (u.is_cuda and u.element_size() == 8 and u.is_contiguous()):
                raise ValueError("states must be contiguous CUDA float64 tensors")
            if u.shape[-2:] != (op.fields, op.grid.n_nodes):
                raise ValueError("state shape does not match its operator")
        self._ops, self._states = list(ops), list(states)
        hs = (C.c_void_p * n)(*[op._h.value for op in ops])
        us = (C.c_void_p * n)(*[u.data_ptr() for u in states])
        rs = (C.c_int * n)(*[1 if u.dim() == 2 else u.shape[0] for u in states])
        self._b = C.c_void_p()
        check(_capi.lib().eo_batch_create(n, hs, us, rs, C.byref(self._b)))

    def apply(self, n_steps=1, stream=None):
        check(_capi.lib().eo_batch_apply(self._b, n_steps, _stream_ptr(stream)))
        return self._states

    def __del__(self):
        if getattr(self, "_b", None) and _capi._lib is not None:
            _capi._lib.eo_batch_destroy(self._b)
            self._b = None
