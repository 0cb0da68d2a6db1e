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


@pytest.mark.parametrize("n_poles,min_X", [(21, 3.0), (57, 10.0), (61, 12.0), (125, 20.0)])
def test_library_fit_meets_contract(capi, n_poles, min_X):
    # the host fitter's output checked by the oracle's brute-force evaluation of
    # eqs. RM_prop1 / RM_prop2 (independent code)
    import paper_1402_5168_gb300 as eo
    from oracle import rational
    alpha, b, X = eo.fit(n_poles)
    assert alpha.size == n_poles and X >= min_X
    band, mod, tail = rational.check_contract(alpha, b, X, 1e-10)
    assert band <= 1e-10 and mod <= 1.0 + 1e-12 and tail < 1.0
    assert np.array_equal(alpha[::-1], np.conj(alpha)) and np.array_equal(b[::-1], np.conj(b))
    assert np.abs(b).max() <= 100.0


def test_every_odd_wide_pole_count_fits(capi):
    # the 64-instance batch draws up to 201 poles; every odd count above 101 (the wide
    # construction) must give an approximant: the last resort adds a zero-residue pair
    # to the next smaller fit, as it does for the dense search below 101
    import paper_1402_5168_gb300 as eo
    for n in range(103, 203, 2):
        alpha, b, X = eo.fit(n)
        assert alpha.size == n and X > 5.0, n


def test_library_fit_for_a_band(capi):
    import paper_1402_5168_gb300 as eo
    from oracle import rational
    alpha, b, X = eo.fit(0, 6.0)
    assert X == 6.0
    band, mod, tail = rational.check_contract(alpha, b, X, 1e-10)
    assert band <= 1e-10 and mod <= 1.0 + 1e-12
    assert alpha.size <= 41


def test_band_between_the_dense_search_and_the_wide_construction(capi):
    # X = 18: no line of the dense search grid up to 101 poles fits it; the wide
    # construction takes over (with more poles) and the contract still holds
    import paper_1402_5168_gb300 as eo
    from oracle import rational
    alpha, b, X = eo.fit(0, 18.0)
    assert X == 18.0
    band, mod, tail = rational.check_contract(alpha, b, X, 1e-10)
    assert band <= 1e-10 and mod <= 1.0 + 1e-12 and tail < 1.0


def test_wide_band_fit_meets_contract(capi):
    # wide band (X = 300): pole line with end corrections, checked by the oracle
    import paper_1402_5168_gb300 as eo
    from oracle import rational
    alpha, b, X = eo.fit(0, 300.0)
    assert X == 300.0 and alpha.size < 4 * 300
    band, mod, tail = rational.check_contract(alpha, b, X, 1e-10)
    assert band <= 1e-10 and mod <= 1.0 + 1e-12 and tail < 1.0
    assert np.array_equal(alpha[::-1], np.conj(alpha)) and np.array_equal(b[::-1], np.conj(b))


def test_batch_create_rejects_empty_and_null(capi):
    L = capi.lib()
    out = C.c_void_p()
    assert L.eo_batch_create(0, None, None, None, C.byref(out)) == 1
    assert L.eo_batch_create(1, None, None, None, C.byref(out)) == 1
    assert L.eo_batch_apply(None, 1, None) == 1
    assert L.eo_batch_destroy(None) == 0


@pytest.mark.parametrize("X,h", [(2 * np.pi * 27.3, 0.18), (60.0, 0.12), (20.0, 0.2)])
def test_library_gaussian_fit_equals_the_oracle_construction(capi, X, h):
    # the library's Sections 3.1-3.2 construction (its own Table 1 copy, C++) against
    # the oracle's (numpy, Table 1 from the golden file), same M
    import paper_1402_5168_gb300 as eo
    from oracle import gauss, rational
    from tests.test_oracle_rational import load_table1
    mu, a = load_table1()
    alpha, b, M = eo.fit_gauss(X, h)
    ao, bo, Mo = gauss.gauss_fit(X, h, mu, a)
    assert M == Mo and alpha.size == ao.size == 2 * (2 * (M + 11) + 1)
    assert np.abs(alpha - ao).max() <= 1e-14 * np.abs(ao).max()
    assert np.abs(b - bo).max() <= 1e-13 * np.abs(bo).max()
    # each line exactly conjugate-closed, and the band contract by brute force
    n1 = alpha.size // 2
    for line in (slice(0, n1), slice(n1, 2 * n1)):
        al, bl = alpha[line], b[line]
        assert np.array_equal(al[::-1], np.conj(al)) and np.array_equal(bl[::-1], np.conj(bl))
    assert gauss.band_error(alpha, b, X) <= 1e-10
    band, mod, _ = rational.check_contract(alpha, b, X, 1e-10)
    assert band <= 1e-10 and mod > 1.0      # eq. RM_prop2 is not part of this construction


def test_gaussian_fit_rejects_bad_arguments(capi):
    L = capi.lib()
    n, M = C.c_int(), C.c_int()
    assert L.eo_fit_gauss(C.c_double(10.0), C.c_double(0.6), C.c_double(1e-10), 0, None, None,
                          C.byref(n), C.byref(M)) == 1
    assert L.eo_fit_gauss(C.c_double(-1.0), C.c_double(0.18), C.c_double(1e-10), 0, None, None,
                          C.byref(n), C.byref(M)) == 1
    assert L.eo_fit_gauss(C.c_double(10.0), C.c_double(0.18), C.c_double(1e-10), 0, None, None,
                          None, None) == 1
    # h too coarse for delta: aliasing e^{-4 pi^2 (1 - 2h)} alone exceeds it
    assert L.eo_fit_gauss(C.c_double(10.0), C.c_double(0.4), C.c_double(1e-10), 0, None, None,
                          C.byref(n), C.byref(M)) == 2
