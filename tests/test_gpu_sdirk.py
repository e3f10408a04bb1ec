"""SDIRK stage solves and SD3/SD4 steps (Sec. 4) on the GPU against the oracle's."""
import numpy as np
import pytest
import torch

from lhcase import Case
from oracle import problems, solver

pytestmark = pytest.mark.gpu

TIGHT = dict(newton_rtol=1e-12, newton_atol=1e-11, gmres_rtol=1e-12, gmres_maxit=400, restart=60)


def _gpu_tg(n, k):
    import paper_2609_16424_b300 as lh
    return lh.Mesh(2, (n, n), (0.0, 0.0), (1.0, 1.0), k, rho0=1.0, gamma=5.0 / 3.0, visc=False, tg_source=True)


def test_stage_solve_matches_oracle_newton():
    """One stage system R(k; tau, u_base) = 0 on a perturbed 2D Q3 state with viscosity;
    u_base is left unchanged and k holds the root."""
    c = Case(2, (3, 3), 3, seed=11, vscale=1.0)
    tau = 0.004
    kref, res = solver.newton(c.hyd, c.u, tau, rtol=1e-12, atol=1e-11)
    assert res.converged
    ub = c.dev(c.u)
    keep = ub.clone()
    kg = torch.zeros_like(ub)
    st = c.gm.stage_solve(ub, kg, tau, **TIGHT)
    assert torch.equal(ub, keep)
    assert st["newton_its"] == st["newton_its_max"] >= 1
    assert max(c.rel_blocks(kg.cpu().numpy(), kref)) <= 1e-9, c.rel_blocks(kg.cpu().numpy(), kref)


@pytest.mark.parametrize("scheme", [3, 4])
def test_sdirk_steps_match_oracle(scheme):
    """Two SD3 / SD4 steps of Taylor-Green Q2-Q1 on 3 x 3 elements, dt = 0.004."""
    hyd, u0 = problems.taylor_green(3, 2, p0=100.0)
    u, kp = u0.copy(), None
    for _ in range(2):
        u, kp, res = solver.sdirk_step(hyd, u, 0.004, scheme, kp, rtol=1e-12, atol=1e-11)
        assert len(res) == 3
    gm = _gpu_tg(3, 2)
    ug = torch.tensor(u0, device="cuda")
    kg = torch.zeros_like(ug)
    for _ in range(2):
        st = gm.sdirk_step(ug, kg, 0.004, scheme=scheme, **TIGHT)
        assert st["newton_its"] >= st["newton_its_max"] >= 1
        assert st["rfinal"] <= 1e-11
    got = ug.cpu().numpy()
    assert np.linalg.norm(got - u) <= 1e-10 * np.linalg.norm(u)
    assert np.linalg.norm(kg.cpu().numpy() - kp) <= 1e-9 * np.linalg.norm(kp)


def test_sd2_step_is_the_newton_step():
    c = Case(2, (5, 4), 3, seed=2, vscale=0.5)
    ua, ka = c.dev(c.u), torch.zeros(c.gm.n, dtype=torch.float64, device="cuda")
    ub, kb = ua.clone(), ka.clone()
    sa = c.gm.newton_step(ua, ka, 0.003, **TIGHT)
    sb = c.gm.sdirk_step(ub, kb, 0.003, scheme=2, **TIGHT)
    assert sa["newton_its"] == sb["newton_its"] == sb["newton_its_max"]
    assert torch.allclose(ua, ub, rtol=1e-13, atol=1e-13) and torch.allclose(ka, kb, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("scheme,lo,hi", [(2, 3.5, 4.6), (3, 7.0, 9.0), (4, 14.0, 28.0)])
def test_sdirk_temporal_order(scheme, lo, hi):
    """Q1-Q0 Taylor-Green on 2 x 2 elements to t = 0.004: halving dt divides the difference
    to a 32-step solution by about 2^p."""
    gm = _gpu_tg(2, 1)
    hyd, u0 = problems.taylor_green(2, 1, p0=100.0)

    def run(nsteps):
        ug = torch.tensor(u0, device="cuda")
        kg = torch.zeros_like(ug)
        for _ in range(nsteps):
            gm.sdirk_step(ug, kg, 0.004 / nsteps, scheme=scheme, **TIGHT)
        return ug.cpu().numpy()
    ref = run(32)
    e = [np.linalg.norm(run(n) - ref) for n in (2, 4)]
    assert lo < e[0] / e[1] < hi, e


def test_sdirk_failures_leave_state_unchanged():
    import paper_2609_16424_b300 as lh
    c = Case(2, (4, 4), 2, seed=5)
    u = c.dev(c.u)
    k = torch.full_like(u, 0.01)
    keep_u, keep_k = u.clone(), k.clone()
    with pytest.raises(lh.LHError) as ei:
        c.gm.sdirk_step(u, k, 0.01, scheme=3, newton_maxit=1, newton_rtol=1e-300, gmres_maxit=2)
    assert ei.value.status == 5        # LH_ENOCONV
    assert ei.value.stats["newton_its"] >= 1
    assert torch.equal(u, keep_u) and torch.equal(k, keep_k)
    for bad in (1, 5):
        with pytest.raises(lh.LHError) as ei:
            c.gm.sdirk_step(u, k, 0.01, scheme=bad)
        assert ei.value.status == 1    # LH_EINVAL
    with pytest.raises(lh.LHError):
        c.gm.stage_solve(u, k, 0.0)
    assert torch.equal(u, keep_u) and torch.equal(k, keep_k)


def test_sd3_time_step_control_follows_the_rule():
    """advance(scheme=3): each attempt follows the Newton-count rule applied to the most
    Newton iterations of one stage."""
    from oracle import solver as osolver
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state
    gm = lh.Mesh(2, (12, 12), (0, 0), (1, 1), 2, gamma=1.4)
    u = blast_state(gm, 0.25)
    dt0 = 4.0 * gm.dt_estimate(u)
    t_end = 25 * dt0
    steps, rejected, hist = gm.advance(u, t_end, fs_cfl=4.0, scheme=3, newton_rtol=1e-5, gmres_rtol=1e-4,
                                       gmres_maxit=200, jvp_prec="fp32")
    assert steps >= 1 and steps == sum(1 for a in hist if a[3]) and rejected == len(hist) - steps
    dt = dt0
    for (c_dt, h, its, accepted) in hist:
        assert abs(c_dt - dt) <= 1e-12 * dt
        dt, ok = osolver.dt_control(dt, 4 if its is None else its)
        assert ok == accepted
    assert sum(h for _, h, _, a in hist if a) == pytest.approx(t_end, rel=1e-12)
    ke, ie = gm.energies(u)
    assert np.isfinite(ke + ie) and ke > 0


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_taylor_green_state_and_l1_error(k):
    """The GPU Taylor-Green initial state equals the oracle's, and the L1 velocity error of
    Sec. 4.1 agrees with the oracle's on the initial and on a moved mesh."""
    from paper_2609_16424_b300.states import taylor_green_problem
    hyd, u0 = problems.taylor_green(3, k, p0=1.0)
    gm, ug = taylor_green_problem(3, k, p0=1.0)
    assert np.allclose(ug.cpu().numpy(), u0, rtol=1e-14, atol=1e-12)
    e_ref = problems.l1_velocity_error(hyd, u0)
    assert abs(gm.tg_velocity_error(ug) - e_ref) <= 1e-12 * max(e_ref, 1e-3)
    u1, _, _ = solver.implicit_midpoint_step(hyd, u0, 0.01, None, rtol=1e-12, atol=1e-11)
    e1 = problems.l1_velocity_error(hyd, u1)
    assert abs(gm.tg_velocity_error(torch.tensor(u1, device="cuda")) - e1) <= 1e-12 * max(e1, 1e-3)


def test_scaled_norm_reaches_the_root_and_tightens_the_v_rows():
    """scaled_norm = 1 (Newton test and GMRES on the row-weighted residual): the stage solve
    reaches the same FP64 root, and at the loose relative tolerance 1e-5 its v and e rows are
    closer to the root than with the plain l2 norm, whose x rows carry no mass factor."""
    from paper_2609_16424_b300.states import taylor_green_problem
    gm, u = taylor_green_problem(16, 3, p0=1.0)
    nx = 2 * gm.NV
    tau = 0.004
    ref = torch.zeros_like(u)
    gm.stage_solve(u, ref, tau, newton_rtol=1e-11, gmres_rtol=1e-12, gmres_maxit=600, restart=60, jvp_prec="fp64")
    tight = torch.zeros_like(u)
    st = gm.stage_solve(u, tight, tau, newton_rtol=1e-11, gmres_rtol=1e-12, gmres_maxit=600, restart=60,
                        jvp_prec="fp64", scaled_norm=1)
    assert st["rfinal"] <= 1e-11 * st["r0"]

    def rel(a, sl):
        return float((a[sl] - ref[sl]).norm() / ref[sl].norm())
    sv, se = slice(nx, 2 * nx), slice(2 * nx, None)
    assert rel(tight, sv) <= 1e-8 and rel(tight, se) <= 1e-8
    errs = {}
    for scaled in (0, 1):
        kk = torch.zeros_like(u)
        gm.stage_solve(u, kk, tau, newton_rtol=1e-5, gmres_rtol=1e-6, gmres_maxit=200, restart=30,
                       jvp_prec="fp32", scaled_norm=scaled)
        errs[scaled] = (rel(kk, sv), rel(kk, se))
    assert errs[1][0] < errs[0][0] and errs[1][0] <= 1e-4, errs


@pytest.mark.parametrize("scheme,lo,hi", [(2, 1.7, 2.3), (3, 2.5, 3.5)])
def test_taylor_green_convergence_rates(scheme, lo, hi):
    """Sec. 4.1 table: Taylor-Green (p0 = 1) to t = 0.5 with Q_k-Q_{k-1} + SD_k (k = scheme),
    dt fixed at 8x the explicit estimate (the paper's FS-CFL 2 step counts), Newton rtol
    1e-9: the L1 velocity error falls at order k between h = 1/32 and 1/64."""
    from paper_2609_16424_b300.states import taylor_green_problem
    errs, steps = [], []
    for inv_h in (32, 64):
        gm, u = taylor_green_problem(inv_h, scheme, p0=1.0)
        n, rej, hist = gm.advance(u, 0.5, fs_cfl=8.0, scheme=scheme, grow=False, max_attempts=400, jvp_prec="fp32",
                                  newton_rtol=1e-9, gmres_rtol=1e-6, gmres_maxit=200, restart=30, newton_maxit=20)
        assert sum(h for _, h, _, a in hist if a) == pytest.approx(0.5, rel=1e-12)
        errs.append(gm.tg_velocity_error(u))
        steps.append(n)
    rate = np.log2(errs[0] / errs[1])
    assert lo < rate < hi, (errs, steps)
