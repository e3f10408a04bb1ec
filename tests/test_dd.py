"""The double-word (float pair) arithmetic of the residual's quadrature-point kernel, checked
on the host against double math (no GPU): the primitives to a few units of 2^-48, the whole
point kernel (stress S, det J, E) to 1e-13 of the size its terms have before the trace and
divergence cancellations that limit any finite precision."""
import ctypes as C

import pytest

BOUNDS = {0: 1e-14, 1: 4e-14, 2: 4e-14, 3: 3e-14, 4: 4e-14, 5: 3e-14, 6: 1e-13, 7: 1e-13, 8: 1e-13, 9: 1e-13}
NAMES = {0: "sum", 1: "product", 2: "quotient", 3: "sqrt", 4: "cbrt", 5: "tanh", 6: "point 2D", 7: "point 2D visc",
         8: "point 3D", 9: "point 3D visc"}


@pytest.mark.parametrize("which", sorted(BOUNDS), ids=[NAMES[w] for w in sorted(BOUNDS)])
def test_double_word_arithmetic(which):
    import paper_2609_16424_b300 as lh
    err = C.c_double()
    assert lh.lib.lh_dd_check(which, 20000, 17, C.byref(err)) == 0
    assert err.value <= BOUNDS[which], err.value
