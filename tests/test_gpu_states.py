"""Problem set-ups built on the GPU (paper_2609_16424_b300/states.py) against the oracle's
(oracle/problems.py): the same state vector and the same materials, so that the residual
of the GPU mesh at the GPU state equals the oracle's residual of its own set-up."""
import numpy as np
import pytest
import torch

import lh_synth
from oracle import problems

pytestmark = pytest.mark.gpu


def _compare(gm, ug, hyd, uo, tau=0.01, seed=3):
    ug = ug.cpu().numpy()
    assert ug.shape == uo.shape
    assert np.abs(ug - uo).max() <= 1e-13 * max(1.0, np.abs(uo).max())
    kk = lh_synth.normal_vector(uo.size, seed, 0.01)
    ref = hyd.residual(uo, kk, tau)
    got = gm.residual(torch.tensor(uo, device="cuda"), torch.tensor(kk, device="cuda"), tau).cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_interface_problem_matches_oracle():
    from paper_2609_16424_b300.states import interface_problem
    gm, ug = interface_problem(14, 6, 3, device="cuda:0")
    hyd, uo = problems.triple_point(14, 6, 3)
    _compare(gm, ug, hyd, uo)


@pytest.mark.parametrize("d,n", [(3, 4), (2, 6)])
def test_blast_state_matches_oracle(d, n):
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state
    gm = lh.Mesh(d, (n,) * d, (0.0,) * d, (1.0,) * d, 2, gamma=1.4, device="cuda:0")
    hyd, uo = problems.sedov(n, 2, d, energy=0.25)
    _compare(gm, blast_state(gm, 0.25), hyd, uo)


@pytest.mark.parametrize("k,p0", [(2, 1.0), (3, 100.0)])
def test_taylor_green_problem_matches_oracle(k, p0):
    from paper_2609_16424_b300.states import taylor_green_problem
    gm, ug = taylor_green_problem(5, k, p0=p0, device="cuda:0")
    hyd, uo = problems.taylor_green(5, k, p0=p0)
    _compare(gm, ug, hyd, uo)
