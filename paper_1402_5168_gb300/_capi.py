"""ctypes declarations of include/expop.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libexpop.so")

EO_OK = 0
STATUS = {0: "EO_OK", 1: "EO_ERR_INVALID_ARG", 2: "EO_ERR_FIT", 3: "EO_ERR_SINGULAR", 4: "EO_ERR_OOM",
          5: "EO_ERR_BUDGET", 6: "EO_ERR_CUDA", 7: "EO_ERR_TIMEOUT", 8: "EO_ERR_UNSUPPORTED"}
STATUS_CODES = {v: k for k, v in STATUS.items()}
WAVE_DIRICHLET, SW_WALLS, WAVE_KAPPA = 0, 1, 2

# every symbol include/expop.h declares
SYMBOLS = ("eo_fit", "eo_grid_create", "eo_grid_create_periodic", "eo_grid_periodic", "eo_grid_info", "eo_grid_nodes", "eo_grid_destroy", "eo_build_operator",
           "eo_get_poles", "eo_memory", "eo_apply", "eo_apply_adjoint", "eo_apply_host", "eo_apply_resolvent", "eo_apply_resolvent_noalloc", "eo_set_timing", "eo_get_timing", "eo_destroy",
           "eo_last_error", "eo_leaf_basis", "eo_batch_create", "eo_batch_apply", "eo_batch_destroy",
           "eo_fit_function", "eo_apply_functions", "eo_fit_gauss", "eo_device_status", "eo_fused_levels",
           "eo_apply_laplacian_filter")


class Opts(C.Structure):
    _fields_ = [("n_poles", C.c_int), ("band", C.c_double), ("tau", C.c_double), ("delta", C.c_double),
                ("sw_f", C.c_double), ("sw_g", C.c_double), ("sw_H", C.c_double), ("precision", C.c_int),
                ("shared_ops", C.c_int), ("max_rhs", C.c_int), ("mem_budget_gb", C.c_double),
                ("fp64_top_levels", C.c_int), ("use_graphs", C.c_int), ("dense_leaves", C.c_int),
                ("autotune", C.c_int), ("sw_consistent", C.c_int), ("fitter", C.c_int),
                ("gauss_h", C.c_double), ("root_dense", C.c_int),
                ("merge_dense", C.c_int), ("tensor_leaves", C.c_int), ("merge_fuse", C.c_int)]


_lib = None


def lib() -> C.CDLL:
    """Load the engine; raises if it was not built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1402_5168_gb300.build_ext.build() first")
    L = C.CDLL(LIB_PATH)
    vp, i64p, dp = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)
    sig = {
        "eo_grid_create": [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                           C.POINTER(vp)],
        "eo_grid_create_periodic": [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.POINTER(vp)],
        "eo_grid_periodic": [vp, C.POINTER(C.c_int)],
        "eo_grid_info": [vp, i64p, i64p, i64p],
        "eo_grid_nodes": [vp, dp, dp],
        "eo_grid_destroy": [vp],
        "eo_build_operator": [vp, C.c_int, dp, C.POINTER(Opts), vp, C.POINTER(vp)],
        "eo_get_poles": [vp, dp, dp, C.POINTER(C.c_int), dp, dp],
        "eo_fit": [C.c_int, C.c_double, C.c_double, C.c_int, dp, dp, C.POINTER(C.c_int), dp],
        "eo_memory": [vp, i64p, i64p],
        "eo_apply": [vp, vp, C.c_int, C.c_int, vp],
        "eo_apply_host": [vp, dp, C.c_int, C.c_int, vp],
        "eo_apply_adjoint": [vp, vp, C.c_int, C.c_int, vp],
        "eo_apply_resolvent": [vp, C.c_int, vp, vp, vp],
        "eo_apply_resolvent_noalloc": [vp, C.c_int, vp, vp, vp],
        "eo_set_timing": [vp, C.c_int],
        "eo_get_timing": [vp, C.POINTER(C.c_int), C.POINTER(C.c_char_p), i64p, dp],
        "eo_destroy": [vp],
        "eo_leaf_basis": [C.c_int, C.c_double, C.c_double, dp, dp, dp],
        "eo_batch_create": [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int), C.POINTER(vp)],
        "eo_batch_apply": [vp, C.c_int, vp],
        "eo_batch_destroy": [vp],
        "eo_fit_function": [vp, C.c_int, C.c_double, dp, dp],
        "eo_apply_functions": [vp, C.c_int, dp, vp, vp, vp],
        "eo_fit_gauss": [C.c_double, C.c_double, C.c_double, C.c_int, dp, dp, C.POINTER(C.c_int),
                         C.POINTER(C.c_int)],
        "eo_fused_levels": [vp, C.c_int, C.POINTER(C.c_int)],
        "eo_apply_laplacian_filter": [vp, dp, vp, C.c_int, C.c_int, vp],
        "eo_device_status": [vp, vp, C.POINTER(C.c_int)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.eo_last_error.argtypes = []
    L.eo_last_error.restype = C.c_char_p
    _lib = L
    return L


class ExpopError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int):
    if status != EO_OK:
        raise ExpopError(status, lib().eo_last_error().decode())
