"""Implicit midpoint Newton-GMRES step on the GPU against the oracle's Newton step."""
import numpy as np
import pytest
import torch

import lh_synth
from lhcase import Case
from oracle import problems, solver

pytestmark = pytest.mark.gpu


def _gpu_tg(n):
    import paper_2609_16424_b300 as lh
    return lh.Mesh(2, (n, n), (0.0, 0.0), (1.0, 1.0), 2, rho0=1.0, gamma=5.0 / 3.0, visc=False, tg_source=True)


def test_taylor_green_ten_steps_match_oracle():
    """Taylor-Green Q2-Q1 on 8x8, dt = 0.01, 10 implicit midpoint steps, Newton rtol 1e-10."""
    hyd, u0 = problems.taylor_green(8, 2, p0=100.0)
    u, kp = u0.copy(), None
    for _ in range(10):
        u, kp, res = solver.implicit_midpoint_step(hyd, u, 0.01, kp, rtol=1e-11, atol=1e-12)
        assert res.converged
    gm = _gpu_tg(8)
    ug = torch.tensor(u0, device="cuda")
    kg = torch.zeros_like(ug)
    for _ in range(10):
        st = gm.newton_step(ug, kg, 0.01, newton_rtol=1e-11, newton_atol=1e-12, gmres_rtol=1e-12,
                             gmres_maxit=300, restart=60)
        assert st["newton_its"] >= 1 and st["rfinal"] <= max(1e-11 * st["r0"], 1e-12)
    got = ug.cpu().numpy()
    assert np.linalg.norm(got - u) <= 1e-10 * np.linalg.norm(u)
    assert abs(problems.l1_velocity_error(hyd, got) - problems.l1_velocity_error(hyd, u)) < 1e-12


def test_blast3d_step_matches_oracle():
    hyd, u0 = problems.sedov(3, 2, 3)
    dt = 0.002
    u1, _, res = solver.implicit_midpoint_step(hyd, u0, dt, None, rtol=1e-11, atol=1e-13)
    assert res.converged
    import paper_2609_16424_b300 as lh
    gm = lh.Mesh(3, (3, 3, 3), (0, 0, 0), (1, 1, 1), 2, rho0=1.0, gamma=1.4)
    ug = torch.tensor(u0, device="cuda")
    st = gm.newton_step(ug, None, dt, newton_rtol=1e-11, newton_atol=1e-13, gmres_rtol=1e-12, gmres_maxit=400,
                        restart=60)
    got = ug.cpu().numpy()
    assert np.linalg.norm(got - u1) <= 1e-9 * np.linalg.norm(u1), st
    # total energy is conserved by the compatible discretisation up to the Newton residual
    ke, ie = gm.energies(ug)
    assert abs(ke + ie - 0.25) <= 1e-9


def test_fp32_jacobian_action_gives_the_fp64_solution():
    """Inexact Newton with an FP32 J.w converges to the same FP64 residual root."""
    c = Case(3, (4, 4, 4), 2, seed=3, vscale=1.0)
    u = c.dev(c.u)
    dt = 0.01
    outs = []
    for prec in ("fp64", "fp32"):
        ug = u.clone()
        kg = torch.zeros_like(ug)
        st = c.gm.newton_step(ug, kg, dt, newton_rtol=1e-11, gmres_rtol=1e-8, gmres_maxit=200, restart=40,
                              jvp_prec=prec)
        outs.append((ug.cpu().numpy(), st))
    (a, sa), (b, sb) = outs
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(a), (sa, sb)


def test_failures_leave_state_unchanged():
    import paper_2609_16424_b300 as lh
    c = Case(2, (4, 4), 2, seed=5)
    u = c.dev(c.u)
    keep = u.clone()
    with pytest.raises(lh.LHError) as ei:
        c.gm.newton_step(u, None, 0.01, newton_maxit=1, newton_rtol=1e-300, gmres_maxit=2)
    assert ei.value.status == 5        # LH_ENOCONV
    assert torch.equal(u, keep)
    # a tangled state is reported, not stepped
    bad = keep.clone()
    bad[:c.gm.NV] = -bad[:c.gm.NV]     # mirror the x coordinate: det J < 0 everywhere
    with pytest.raises(lh.LHError) as ei:
        c.gm.newton_step(bad, None, 0.01)
    assert ei.value.status == 4        # LH_ETANGLED
    with pytest.raises(ValueError):
        c.gm.residual(u[:-1].contiguous(), u, 0.1)


def test_autograd_function():
    import paper_2609_16424_b300 as lh
    c = Case(2, (3, 3), 2, seed=8)
    u = c.dev(c.u)
    k = c.dev(lh_synth.normal_vector(c.gm.n, 1, 0.1)).requires_grad_(True)
    y = c.dev(lh_synth.normal_vector(c.gm.n, 2))
    tau = 0.02
    r = lh.StageResidual.apply(k, u, tau, c.gm)
    (g,) = torch.autograd.grad((r * y).sum(), k)
    assert torch.allclose(g, c.gm.jtvp(u, k.detach(), tau, y), rtol=0, atol=1e-13 * g.abs().max().item())
    import torch.autograd.forward_ad as fwAD
    dk = c.dev(lh_synth.normal_vector(c.gm.n, 3))
    with fwAD.dual_level():
        kd = fwAD.make_dual(k.detach(), dk)
        out = lh.StageResidual.apply(kd, u, tau, c.gm)
        tangent = fwAD.unpack_dual(out).tangent
    ref = c.hyd.jvp_complex_step(c.u, k.detach().cpu().numpy(), tau, dk.cpu().numpy())
    assert np.linalg.norm(tangent.cpu().numpy() - ref) <= 1e-11 * np.linalg.norm(ref)


def test_dt_estimate_closed_form():
    """Undeformed box, v = 0, uniform e: dt = (h/k) / (c_s + mu / (rho h/k)) with
    mu = rho h0 (q2 ds + q1 c_s / 2) (psi(0) = 1/2, |0|_ds = ds, ds = 2 c_s h/h_coarse)."""
    import paper_2609_16424_b300 as lh
    gm = lh.Mesh(2, (4, 4), (0, 0), (1, 1), 2, gamma=1.4)
    x0 = gm.initial_nodes()
    u = torch.zeros(gm.n, dtype=torch.float64, device="cuda")
    u[:x0.numel()] = x0
    u[2 * x0.numel():] = 2.0
    ep = 0.5 * (2.0 + np.sqrt(4.0 + 1e-12))
    cs = np.sqrt(1.4 * 0.4 * ep)
    h = 0.25
    mu = 1.0 * h * (1.0 * 2 * cs + 0.5 * cs * 0.5)
    hm = h / 2
    assert abs(gm.dt_estimate(u) - hm / (cs + mu / hm)) <= 1e-12


def test_time_step_control_follows_the_rule():
    """advance(): every attempt follows the Newton-count rule of oracle.solver.dt_control
    (<= 1 iteration: x1.05; 2-3: keep; >= 4 or failure: reject, x0.85)."""
    from oracle import solver as osolver
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state
    gm = lh.Mesh(3, (6, 6, 6), (0,) * 3, (1,) * 3, 2, gamma=1.4)
    u = blast_state(gm, 0.25)
    dt0 = 2.0 * gm.dt_estimate(u)
    t_end = 40 * dt0
    steps, rejected, hist = gm.advance(u, t_end, fs_cfl=2.0, newton_rtol=1e-5, gmres_rtol=1e-4,
                                       gmres_maxit=200, jvp_prec="fp32")
    assert abs(hist[0][0] - dt0) <= 1e-15 * dt0
    assert steps == sum(1 for a in hist if a[3]) and rejected == len(hist) - steps
    dt = dt0
    for (c_dt, h, its, accepted) in hist:
        assert abs(c_dt - dt) <= 1e-12 * dt
        dt, ok = osolver.dt_control(dt, 4 if its is None else its)
        assert ok == accepted
    assert sum(h for _, h, _, a in hist if a) == pytest.approx(t_end, rel=1e-12)


def test_adaptive_forcing_reaches_the_same_root():
    """Eisenstat-Walker forcing terms change the linear tolerances, not the Newton root."""
    c = Case(3, (4, 4, 4), 2, seed=3, vscale=1.0)
    u = c.dev(c.u)
    outs = []
    for forcing in (0, 1):
        ug, kg = u.clone(), torch.zeros_like(u)
        st = c.gm.newton_step(ug, kg, 0.01, newton_rtol=1e-10, gmres_rtol=1e-8, gmres_maxit=300, restart=40,
                              jvp_prec="fp32", forcing=forcing, eta_max=0.1)
        assert st["rfinal"] <= 1e-10 * st["r0"]
        outs.append((ug.cpu().numpy(), st))
    (a, sa), (b, sb) = outs
    assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(a), (sa, sb)
    import paper_2609_16424_b300 as lh
    with pytest.raises(lh.LHError):
        c.gm.newton_step(u.clone(), None, 0.01, forcing=1, eta_max=1.5)
