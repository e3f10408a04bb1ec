"""The linearisation record of the reduced-precision Jacobian actions (no GPU): the tangent
formed from the record equals the dual-number tangent of the point kernel (the same kernel
the GPU parity tests pin against the oracle's complex-step derivative) to rounding in
double, and to float rounding when record and tangent are float, as on the GPU."""
import ctypes as C

import pytest


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("visc", [0, 1])
def test_record_tangent_matches_dual_tangent(dim, visc):
    import paper_2609_16424_b300 as lh
    md, mf = C.c_double(), C.c_double()
    assert lh.lib.lh_qp_tangent_check(dim, visc, 2000, 7, C.byref(md), C.byref(mf)) == 0
    assert md.value <= 1e-10, md.value
    assert mf.value <= 1e-6, mf.value


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("visc", [0, 1])
def test_record_adjoint_is_the_transpose(dim, visc):
    """<L x, y> = <x, L^T y> for the linearised point map and its hand-written transpose."""
    import paper_2609_16424_b300 as lh
    worst = C.c_double()
    assert lh.lib.lh_qp_adjoint_check(dim, visc, 2000, 3, C.byref(worst)) == 0
    assert worst.value <= 1e-13, worst.value
