"""Pins of the oracle's Newton solve and implicit midpoint step."""
import numpy as np
import pytest

import lh_synth
from oracle import problems, solver
from oracle.fem import Mesh
from oracle.hydro import Hydro, Params, jacobian_sparse


def _energy(hyd, u):
    return hyd.kinetic_energy(u) + hyd.internal_energy(u)


def test_sparse_jacobian_equals_dense():
    hyd, u = problems.taylor_green(3, 2, p0=100.0)
    k = lh_synth.normal_vector(u.size, 0, 0.1)
    Jd = hyd.jacobian(u, k, 0.01)
    Js = jacobian_sparse(hyd, u, k, 0.01).toarray()
    assert np.array_equal(Jd, Js)


@pytest.mark.parametrize("d,n,k", [(2, 4, 2), (3, 2, 1)])
def test_total_energy_conserved_by_midpoint(d, n, k):
    """Compatible discretisation (Eqs. (6a)-(7)): with R(k) = 0 the implicit midpoint
    step changes 1/2 v^T M_V v + 1^T M_E e by dt (r_v^T w_v + 1^T r_e) = 0, so the total
    energy changes only by the Newton residual (here 1e-12 relative)."""
    hyd, u = problems.sedov(n, k, d, energy=0.25)
    E0 = _energy(hyd, u)
    assert abs(E0 - 0.25) < 1e-12
    kp = None
    for _ in range(2):
        u, kp, res = solver.implicit_midpoint_step(hyd, u, 0.002, kp, rtol=1e-13, atol=1e-15)
        assert res.converged
    assert abs(_energy(hyd, u) - E0) < 1e-10 * E0
    # mass is exactly conserved (m_q fixed), and the blast moved something
    assert np.abs(hyd.m.split(u)[1]).max() > 1e-3


def test_blast_symmetry_2d():
    """Corner deposit with walls on a square: the solution is symmetric under x <-> y."""
    hyd, u = problems.sedov(4, 2, 2)
    u, _, res = solver.implicit_midpoint_step(hyd, u, 0.003, None)
    assert res.converged
    m = hyd.m
    x, v, e = m.split(u)
    lat = m.lat[0]
    perm = np.arange(m.NV).reshape(lat, lat).T.ravel()        # swap lattice axes
    assert np.allclose(x[0], x[1][perm], atol=1e-12)
    assert np.allclose(v[0], v[1][perm], atol=1e-12)
    eperm = np.arange(m.NE).reshape(4, 4).T.ravel()
    lperm = np.arange(m.NL).reshape(m.L, m.L).T.ravel()
    assert np.allclose(e, e[eperm][:, lperm], atol=1e-10)


def test_midpoint_is_second_order_in_time():
    """Implicit midpoint (SD2, Sec. 4.1) is second order: halving dt divides the
    difference to a fine-step solution by about 4."""
    def run(nsteps):
        hyd, u = problems.taylor_green(2, 2, p0=100.0)
        kp = None
        for _ in range(nsteps):
            u, kp, _ = solver.implicit_midpoint_step(hyd, u, 0.01 / nsteps, kp, rtol=1e-13)
        return u
    ref = run(32)
    e1 = np.linalg.norm(run(2) - ref)
    e2 = np.linalg.norm(run(4) - ref)
    assert 3.5 < e1 / e2 < 4.5


def test_newton_converges_and_line_search_keeps_mesh_valid():
    m = Mesh((3, 3), (0.0, 0.0), (1.0, 1.0), 2)
    hyd = Hydro(m, Params(m, gamma=1.4, visc=True))
    u = problems.perturbed_state(hyd, lh_synth.perturbed_draws((3, 3), 2, 7), vscale=5.0)
    k, res = solver.newton(hyd, u, 0.02, rtol=1e-10)
    assert res.converged
    assert np.linalg.norm(hyd.residual(u, k, 0.02)) <= 1e-10 * res.r0
    assert hyd.min_detj(m.split(u + 0.02 * k)[0]) > 0


def test_dt_control_rule():
    """Sec. 4: <= 1 Newton iteration: dt x 1.05; 2-3: keep; >= 4: reject and use 0.85 dt."""
    assert solver.dt_control(1.0, 0) == (1.05, True)
    assert solver.dt_control(1.0, 1) == (1.05, True)
    assert solver.dt_control(1.0, 3) == (1.0, True)
    assert solver.dt_control(1.0, 4) == (0.85, False)


@pytest.mark.slow
def test_taylor_green_spatial_rate():
    """Q2-Q1 Taylor-Green: the L1 velocity error falls at about second order or better
    under refinement (Table 1 reports rates 1.9-2.5 for Q2Q1 + SD2)."""
    errs = []
    for n in (4, 8):
        hyd, u = problems.taylor_green(n, 2, p0=100.0)
        kp = None
        for _ in range(8):
            u, kp, _ = solver.implicit_midpoint_step(hyd, u, 0.025, kp)
        errs.append(problems.l1_velocity_error(hyd, u))
    rate = np.log2(errs[0] / errs[1])
    assert rate > 1.9, errs


def test_velocity_block_diagonal():
    """diag(dR_v/dk_v) equals central differences of the residual, one velocity unknown at
    a time; at tau = 0 it is the diagonal of M_V (1 on the fixed rows)."""
    m = Mesh((2, 2), (0.0, 0.0), (1.0, 1.0), 2)
    hyd = Hydro(m, Params(m, gamma=1.4, visc=True))
    u = problems.perturbed_state(hyd, lh_synth.perturbed_draws((2, 2), 2, 4), vscale=3.0)
    k = lh_synth.normal_vector(u.size, 1, 0.5)
    tau = 0.01
    d = solver.velocity_block_diagonal(hyd, u, k, tau)
    n1 = m.d * m.NV
    h = 1e-6
    fd = np.empty(n1)
    for i in range(n1):
        e = np.zeros(u.size)
        e[n1 + i] = h
        fd[i] = (hyd.residual(u, k + e, tau)[n1 + i] - hyd.residual(u, k - e, tau)[n1 + i]) / (2 * h)
    assert np.allclose(d, fd, rtol=1e-6, atol=1e-9 * np.abs(d).max())
    d0 = solver.velocity_block_diagonal(hyd, u, k, 0.0)
    mv = np.tile(hyd.mass_v_sparse().diagonal(), m.d)
    free = ~hyd.fixed.ravel()
    assert np.allclose(d0[free], mv[free], rtol=1e-13)
    assert np.all(d0[~free] == 1.0) and np.all(d[~free] == 1.0)
    # the viscous term changes the free rows at tau > 0
    assert np.abs(d - d0)[free].max() > 1e-6 * np.abs(d0).max()
