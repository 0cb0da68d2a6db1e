"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every symbol include/expop.h declares, reproduces the public node numbering,
and rejects bad arguments with status codes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import sem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "expop.h")


@pytest.fixture(scope="module")
def capi():
    from paper_1402_5168_gb300 import _capi, build_ext
    if not os.path.exists(_capi.LIB_PATH):
        build_ext.build()
    return _capi


def test_every_declared_symbol_is_exported(capi):
    text = open(HEADER).read()
    declared = set(re.findall(r"^\s*(?:eo_status|const char \*)\s*(eo_\w+)\s*\(", text, re.M))
    assert declared == set(capi.SYMBOLS)
    L = capi.lib()
    for name in declared:
        assert hasattr(L, name)


@pytest.mark.parametrize("nlx,nly,p", [(4, 4, 12), (2, 8, 7), (1, 1, 5)])
def test_node_numbering_matches_oracle(capi, nlx, nly, p):
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(nlx, nly, p)
    x, y = g.nodes()
    og = sem.Grid(nlx, nly, p)
    assert g.n_nodes == og.n_nodes and g.n_interior == og.n_int
    assert np.array_equal(x, og.x) and np.array_equal(y, og.y)


def test_bad_arguments_are_rejected(capi):
    L = capi.lib()
    h = C.c_void_p()
    assert L.eo_grid_create(3, 4, 12, 0.0, 1.0, 0.0, 1.0, C.byref(h)) == 1     # not a power of two
    assert b"power" in L.eo_last_error()
    assert L.eo_grid_create(4, 4, 3, 0.0, 1.0, 0.0, 1.0, C.byref(h)) == 1      # p too small
    assert L.eo_grid_create(4, 4, 8, 1.0, 0.0, 0.0, 1.0, C.byref(h)) == 1      # empty domain
    assert L.eo_grid_info(None, None, None, None) == 1
    assert L.eo_apply(None, None, 1, 1, None) == 1
    assert L.eo_destroy(None) == 0
