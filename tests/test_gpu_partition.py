"""Two-slab decomposition emulated on one GPU: residual and Jacobian actions with one halo
exchange equal the unpartitioned operators (the only difference is the grouping of the
sums on the cut plane), and the oracle."""
import numpy as np
import pytest
import torch

import lh_synth
from lhcase import Case

pytestmark = pytest.mark.gpu

CASES = [(3, (3, 4, 5), 2, 2), (3, (4, 3, 4), 1, 1), (2, (6, 5), 3, 2), (2, (5, 7), 2, 5)]
IDS = [f"d{c[0]}_n{'x'.join(map(str, c[1]))}_k{c[2]}_cut{c[3]}" for c in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def setup(request):
    from paper_2609_16424_b300.partition import SlabPair
    dim, n, k, cut = request.param
    c = Case(dim, n, k, seed=41)
    sp = SlabPair(dim, n, (0.0,) * dim, (1.0,) * dim, k, cut, gamma=1.4)
    return c, sp


def _rel(c, a, b):
    return max(c.rel_blocks(a.double().cpu().numpy(), b.double().cpu().numpy()))


def test_partitioned_residual(setup):
    c, sp = setup
    u = c.dev(c.u)
    kk = c.dev(lh_synth.normal_vector(c.gm.n, 1, 0.05))
    tau = 0.01
    r = sp.residual(u, kk, tau)
    assert _rel(c, r, c.gm.residual(u, kk, tau)) <= 1e-13
    ref = c.hyd.residual(c.u, kk.cpu().numpy(), tau)
    assert max(c.rel_blocks(r.cpu().numpy(), ref)) <= 1e-12


def test_partitioned_jvp(setup):
    c, sp = setup
    u = c.dev(c.u)
    kk = c.dev(lh_synth.normal_vector(c.gm.n, 2, 0.05))
    dk = c.dev(lh_synth.normal_vector(c.gm.n, 3))
    tau = 0.01
    assert _rel(c, sp.jvp(u, kk, tau, dk), c.gm.jvp(u, kk, tau, dk)) <= 1e-13
    dkf = dk.float()
    c.gm.linearize(u, kk, tau)
    assert _rel(c, sp.jvp_record(u, kk, tau, dkf), c.gm.jvp(u, kk, tau, dkf, lin=True)) <= 1e-6
    if c.dim == 2 or c.k <= 2:
        assert _rel(c, sp.jvp_record(u, kk, tau, dkf, tc="bf16"), c.gm.jvp(u, kk, tau, dkf, tc="bf16")) <= 1e-6


def test_partition_interface_copies_agree(setup):
    """After the exchange both sides hold bit-identical values on the cut plane."""
    c, sp = setup
    u = c.dev(c.u)
    kk = c.dev(lh_synth.normal_vector(c.gm.n, 4, 0.05))
    parts = sp.exchange([m.residual(a, b, 0.01) for m, a, b in zip(sp.parts, sp.split(u), sp.split(kk))])
    g0 = torch.zeros(sp.n_g, dtype=torch.float64, device="cuda")
    g1 = torch.zeros_like(g0)
    g0[sp.rows[0]] = parts[0]
    g1[sp.rows[1]] = parts[1]
    both = torch.zeros(sp.n_g, dtype=torch.bool, device="cuda")
    both[sp.rows[0]] = True
    m1 = torch.zeros_like(both)
    m1[sp.rows[1]] = True
    both &= m1
    assert both.sum() > 0 and torch.equal(g0[both], g1[both])


def test_partitioned_energies_and_dt(setup):
    c, sp = setup
    u = c.dev(c.u)
    ke, ie = sp.energies(u)
    kg, ig = c.gm.energies(u)
    assert abs(ke - kg) <= 1e-13 * abs(kg) and abs(ie - ig) <= 1e-13 * abs(ig)
    assert sp.dt_estimate(u) == pytest.approx(c.gm.dt_estimate(u), rel=1e-14)
