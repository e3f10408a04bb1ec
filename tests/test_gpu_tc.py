"""Tensor-core J.w (TF32 / BF16 operands, FP32 accumulation) against the oracle.

The direction is rounded to float as the kernels see it; the reference is the oracle's
complex-step J.dk of that float direction.  Bounds per block (x, v, e rows), relative L2:
five unit roundoffs of the operand format, 5 * 2^-11 (TF32, 10-bit mantissa) and
5 * 2^-9 (BF16, 7-bit mantissa).  The x rows (dk_x - tau dk_v) do not pass through the
tensor cores and keep the FP32 bound.
"""
import numpy as np
import pytest
import torch

import lh_synth
from lhcase import Case

pytestmark = pytest.mark.gpu

TOL = {"tf32": 5 * 2.0 ** -11, "bf16": 5 * 2.0 ** -9}

CASES = [
    (2, (7, 5), 1, True, False),
    (2, (7, 5), 2, True, False),
    (2, (5, 3), 2, False, True),      # Taylor-Green source, no viscosity
    (2, (4, 3), 3, True, False),
    (2, (3, 2), 4, True, False),
    (3, (5, 4, 3), 1, True, False),
    (3, (3, 3, 3), 2, True, False),
    (2, (61, 50), 2, True, False),    # 3050 elements: 191 batches of 16, > 1 batch per CTA
    (3, (9, 8, 7), 2, True, False),   # 504 elements, ragged last batch (8 of 16)
]
IDS = [f"d{c[0]}_n{'x'.join(map(str, c[1]))}_k{c[2]}{'_visc' if c[3] else ''}{'_tg' if c[4] else ''}" for c in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request):
    dim, n, k, visc, tg = request.param
    return Case(dim, n, k, seed=21, visc=visc, tg=tg)


def _tc_jvp(case, kind, tau=0.02, seed=4, kscale=0.1):
    # k scaled with the element size so that w = u + tau k stays untangled on fine meshes
    kk = lh_synth.normal_vector(case.gm.n, seed, min(kscale, 5 * kscale / max(case.n)))
    dk = lh_synth.normal_vector(case.gm.n, seed + 1).astype(np.float32).astype(np.float64)
    ref = case.hyd.jvp_complex_step(case.u, kk, tau, dk)
    assert np.all(np.isfinite(ref)), "invalid input: the oracle's J.dk is not finite (tangled w)"
    u, kd = case.dev(case.u), case.dev(kk)
    case.gm.linearize(u, kd, tau)
    got = case.gm.jvp(u, kd, tau, case.dev(dk, torch.float32), tc=kind).double().cpu().numpy()
    case.gm.tc_status()
    return case.rel_blocks(got, ref)


@pytest.mark.parametrize("kind", ["tf32", "bf16"])
def test_jvp_tc_parity(case, kind):
    rel = _tc_jvp(case, kind)
    assert rel[0] <= 2e-5, rel
    assert max(rel[1:]) <= TOL[kind], rel


def test_jvp_tc_larger_tau(case):
    """tau = 0.2 weights the force tangent ten times more against the mass terms (k scaled
    down so that w = u + tau k stays untangled)."""
    rel = _tc_jvp(case, "tf32", tau=0.2, seed=7, kscale=0.01)
    assert rel[0] <= 2e-5, rel
    assert max(rel[1:]) <= TOL["tf32"], rel


def test_jvp_tc_unsupported_orders_are_refused():
    import paper_2609_16424_b300 as lh
    c = Case(3, (1, 1, 2), 3, seed=2)
    u = c.dev(c.u)
    k = torch.zeros_like(u)
    c.gm.linearize(u, k, 0.01)
    with pytest.raises(lh.LHError) as ei:
        c.gm.jvp(u, k, 0.01, torch.zeros(c.gm.n, dtype=torch.float32, device="cuda"), tc="tf32")
    assert ei.value.status == 1
    with pytest.raises(lh.LHError):
        c.gm.newton_step(u.clone(), None, 0.01, jvp_prec="bf16")


@pytest.mark.parametrize("kind", ["tf32", "bf16"])
def test_tc_newton_gives_the_fp64_solution(kind):
    """Inexact Newton with a tensor-core J.w converges to the same FP64 residual root."""
    c = Case(3, (4, 4, 4), 2, seed=3, vscale=1.0)
    u = c.dev(c.u)
    dt = 0.01
    outs = []
    for prec in ("fp64", kind):
        ug = u.clone()
        kg = torch.zeros_like(ug)
        st = c.gm.newton_step(ug, kg, dt, newton_rtol=1e-11, gmres_rtol=1e-8, gmres_maxit=200, restart=40,
                              jvp_prec=prec)
        outs.append((ug.cpu().numpy(), st))
    (a, sa), (b, sb) = outs
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(a), (sa, sb)
    c.gm.tc_status()


@pytest.mark.parametrize("dim,n,k", [(3, (24, 24, 24), 2), (2, (80, 70), 3), (2, (60, 60), 4)])
def test_tc_many_batches_per_cta(dim, n, k):
    """Persistent CTAs that process several batches, each with several sub-chunks of
    quadrature points (the pipelined forward MMAs): the tensor-core J.w agrees with the
    FP32 record J.w (itself checked against the oracle) and no bounded wait expires."""
    import paper_2609_16424_b300 as lh
    import lh_synth
    gm = lh.Mesh(dim, n, (0.0,) * dim, (1.0,) * dim, k, gamma=1.4)
    x0 = gm.initial_nodes()
    u = torch.zeros(gm.n, dtype=torch.float64, device="cuda")
    u[:x0.numel()] = x0
    u[dim * gm.NV:2 * dim * gm.NV] = torch.tensor(lh_synth.normal_vector(dim * gm.NV, 11, 0.1), device="cuda")
    u[2 * dim * gm.NV:] = 1.0
    kk = torch.zeros_like(u)
    tau = 1e-3
    gm.linearize(u, kk, tau)
    dk = torch.tensor(lh_synth.normal_vector(gm.n, 12), dtype=torch.float32, device="cuda")
    ref = gm.jvp(u, kk, tau, dk, lin=True).double()
    nx = dim * gm.NV
    for kind in ("tf32", "bf16"):
        got = gm.jvp(u, kk, tau, dk, tc=kind).double()
        gm.tc_status()
        for sl in (slice(nx, 2 * nx), slice(2 * nx, gm.n)):
            assert float((got[sl] - ref[sl]).norm() / ref[sl].norm()) <= TOL[kind]


@pytest.mark.parametrize("kind", ["tf32", "bf16"])
def test_tc_wait_limit_reports_and_returns(kind):
    """A tensor-core wait that runs out does not hang the launch: with a poll limit of 0 the
    first wait on an MMA completion gives up, every later wait of the launch is skipped (no
    cascade of full-length waits over the batches a CTA owns), the element rows come back
    NaN, lh_tc_status reports LH_ECUDA, and the next launch with the default limit is
    correct again (the context stays usable)."""
    import time
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.hydro import LHError
    c = Case(2, (61, 50), 2, seed=21, visc=True)       # 191 batches: several per CTA
    kk = lh_synth.normal_vector(c.gm.n, 4, 0.1 * 5 / 61)
    dk = lh_synth.normal_vector(c.gm.n, 5).astype(np.float32)
    u, kd = c.dev(c.u), c.dev(kk)
    tau = 0.02
    c.gm.linearize(u, kd, tau)
    good = c.gm.jvp(u, kd, tau, c.dev(dk, torch.float32), tc=kind).cpu().numpy()
    c.gm.tc_status()
    prev = lh.lib.lh_tc_set_wait_polls(0)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bad = c.gm.jvp(u, kd, tau, c.dev(dk, torch.float32), tc=kind).cpu().numpy()
        took = time.perf_counter() - t0
    finally:
        lh.lib.lh_tc_set_wait_polls(prev)
    assert took < 5.0, took
    assert np.isnan(bad[c.nx:]).any()
    with pytest.raises(LHError):
        c.gm.tc_status()
    again = c.gm.jvp(u, kd, tau, c.dev(dk, torch.float32), tc=kind).cpu().numpy()
    c.gm.tc_status()
    assert np.array_equal(again, good)
