"""The library's SDIRK tableaux (computed in C++ independently of the oracle) meet the
Runge-Kutta order conditions of SD2/SD3/SD4 (Sec. 4) and equal the oracle's.  Host only."""
import ctypes as C

import numpy as np
import pytest

from oracle import solver


def _lib_tableau(scheme):
    import paper_2609_16424_b300 as lh
    s = C.c_int()
    A = (C.c_double * 9)()
    b = (C.c_double * 3)()
    st = lh.lib.lh_sdirk_tableau(scheme, C.byref(s), A, b)
    assert st == 0
    n = s.value
    return np.array(A[:]).reshape(3, 3)[:n, :n], np.array(b[:n])


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_library_tableau_order_conditions(scheme):
    A, b = _lib_tableau(scheme)
    c = A.sum(axis=1)
    conds = [(1, b.sum(), 1.0), (2, b @ c, 0.5), (3, b @ c**2, 1 / 3), (3, b @ (A @ c), 1 / 6),
             (4, b @ c**3, 0.25), (4, b @ (c * (A @ c)), 1 / 8), (4, b @ (A @ c**2), 1 / 12),
             (4, b @ (A @ (A @ c)), 1 / 24)]
    for order, val, want in conds:
        if order <= scheme:
            assert abs(val - want) < 1e-14, (order, val, want)
    assert np.allclose(np.triu(A, 1), 0.0) and np.allclose(np.diag(A), A[0, 0])
    Ao, bo = solver.sdirk_tableau(scheme)
    # gamma of SD3 is a root of a cubic: numpy.roots and the library's Newton iteration agree to a few ulp
    assert np.allclose(A, Ao, rtol=0, atol=1e-14) and np.allclose(b, bo, rtol=0, atol=1e-14)


def test_library_tableau_rejects_other_schemes():
    import paper_2609_16424_b300 as lh
    s = C.c_int()
    A = (C.c_double * 9)()
    b = (C.c_double * 3)()
    for bad in (1, 5):
        assert lh.lib.lh_sdirk_tableau(bad, C.byref(s), A, b) == 1
