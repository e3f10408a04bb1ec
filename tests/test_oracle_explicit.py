"""Pins of the oracle's explicit path (oracle/explicit.py) and of the original tensor
viscosity mu_exp (oracle/hydro.py stress_exp): order conditions and stability polynomials
of the Runge-Kutta tableaux, exact total-energy conservation of the RK2-average scheme,
temporal orders 2 / 3 / 4 on the Taylor-Green vortex, momentum conservation, and closed
forms of mu_exp where its eigen-decomposition is known."""
import math

import numpy as np
import pytest

import lh_synth
from oracle import problems
from oracle.explicit import RK_TABLEAUX, Explicit, explicit_advance, explicit_step, rk_step, total_energy
from oracle.fem import Mesh
from oracle.hydro import Hydro, Params, stress_exp


# -- Runge-Kutta tableaux -----------------------------------------------------------------
def test_rk_order_conditions():
    """Butcher's order conditions: RK3 SSP meets those of order 3, RK4 those of order 4."""
    for p, (A, b) in RK_TABLEAUX.items():
        c = A.sum(axis=1)
        conds = [b.sum() - 1, b @ c - 1 / 2, b @ c ** 2 - 1 / 3, b @ (A @ c) - 1 / 6]
        if p == 4:
            conds += [b @ c ** 3 - 1 / 4, b @ (c * (A @ c)) - 1 / 8, b @ (A @ c ** 2) - 1 / 12,
                      b @ (A @ (A @ c)) - 1 / 24]
        assert max(abs(x) for x in conds) < 1e-15, (p, conds)
        assert np.allclose(np.triu(A), 0.0)          # explicit


@pytest.mark.parametrize("p", [3, 4])
def test_rk_stability_polynomial(p):
    """On y' = lam y one step multiplies y by sum_{j<=p} z^j / j! (z = lam dt) for p <= 4."""
    A, b = RK_TABLEAUX[p]
    for z in (-0.3, -1.7, 0.4 + 0.9j, -2.5j):
        y = rk_step(lambda v: z * v, np.array([1.0 + 0j]), 1.0, A, b)
        ref = sum(z ** j / math.factorial(j) for j in range(p + 1))
        assert abs(y[0] - ref) < 1e-14


# -- explicit hydro steps -------------------------------------------------------------------
def _blast(n=3, k=2, d=2, model='imp'):
    m = Mesh((n,) * d, (0.0,) * d, (1.0,) * d, k)
    hyd = Hydro(m, Params(m, gamma=1.4, visc=True, visc_model=model))
    e = np.zeros((m.NE, m.NL)) + 0.01
    e[0, :] = 0.5 * m.NE
    u = m.join(hyd.x0, np.zeros((d, m.NV)), e)
    return hyd, u


@pytest.mark.parametrize("model", ["imp", "exp"])
@pytest.mark.parametrize("d", [2, 3])
def test_rk2_average_conserves_total_energy(model, d):
    """Compatible discretisation + RK2-average: the kinetic change -dt vbar^T F.1 and the
    internal change +dt vbar^T F.1 cancel exactly (no source), for either viscosity."""
    hyd, u = _blast(3 if d == 2 else 2, 2, d, model)
    E0 = total_energy(hyd, u)
    u, steps, _ = explicit_advance(hyd, u, 0.05, 0.3, 2)     # with the explicit step control
    assert steps >= 2
    assert abs(total_energy(hyd, u) - E0) <= 1e-14 * E0
    assert np.abs(hyd.m.split(u)[1]).max() > 0.1          # the blast moved


def test_momentum_is_conserved_without_walls():
    """Partition of unity: sum_i (F.1)_{c,i} = 0, so M_V a sums to zero per component and the
    total momentum sum_i (M_V v)_{c,i} is unchanged by any explicit step."""
    m = Mesh((3, 2), (0.0, 0.0), (1.0, 1.0), 2)
    hyd = Hydro(m, Params(m, gamma=1.4, visc=True, bc_mask=0))
    u = problems.perturbed_state(hyd, lh_synth.perturbed_draws((3, 2), 2, 4))
    ex = Explicit(hyd)

    def momentum(w):
        return hyd.apply_mass_v(m.split(w)[1]).sum(axis=1)
    p0 = momentum(u)
    for scheme in (2, 3, 4):
        u1 = explicit_step(ex, u, 1e-3, scheme)
        assert np.abs(momentum(u1) - p0).max() <= 1e-13 * (1 + np.abs(p0).max())


@pytest.mark.parametrize("scheme,order", [(2, 2), (3, 3), (4, 4)])
def test_temporal_order_on_taylor_green(scheme, order):
    """Errors against a fine RK4 reference fall as dt^order (Taylor-Green, 4 x 4 Q2, t = 0.06)."""
    hyd, u0 = problems.taylor_green(4, 2, p0=1.0)
    ex = Explicit(hyd)
    t_end = 0.06

    def run(s, nsteps):
        u = u0.copy()
        for _ in range(nsteps):
            u = explicit_step(ex, u, t_end / nsteps, s)
        return u
    ref = run(4, 96)
    errs = [np.linalg.norm(run(scheme, n) - ref) for n in (3, 6)]
    rate = math.log2(errs[0] / errs[1])
    assert rate > order - 0.35, (errs, rate)


# -- mu_exp -----------------------------------------------------------------------------------
def _prm(d, vorticity=False):
    m = Mesh((1,) * d, (0.0,) * d, (1.0,) * d, 2)
    prm = Params(m, visc=True, visc_model='exp', h0=0.1, vorticity=vorticity)
    return prm


def _mu_exp(grad_v, J, J0inv, rho=1.3, e=2.0, gam=1.4, vorticity=False):
    d = grad_v.shape[0]
    prm = _prm(d, vorticity)
    sig, mu = stress_exp(grad_v, J, J0inv, np.array(rho), np.array(e), np.array(gam), prm, d, return_mu=True)
    return sig, float(mu), prm


def _rot(d, a):
    if d == 2:
        return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    c, s = np.cos(a), np.sin(a)
    Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
    Rx = np.array([[1.0, 0, 0], [0, np.cos(2 * a), -np.sin(2 * a)], [0, np.sin(2 * a), np.cos(2 * a)]])
    return Rz @ Rx


@pytest.mark.parametrize("d", [2, 3])
def test_mu_exp_principal_axes(d):
    """eps(v) = R diag(lam) R^T on an undeformed (rotated) element: l = l0, lambda_1 = min lam,
    mu = rho (q2 l0^2 |lambda_1| + q1 l0 c_s) under compression (psi_1 = 1), and
    sigma = -p I + mu eps(v) rotates with R."""
    lam = np.array([-0.7, 0.2, 0.5])[:d]
    R = _rot(d, 0.37)
    G = R @ np.diag(lam) @ R.T
    J0 = np.eye(d) * 0.25
    J = R @ J0                                     # rigidly rotated element: J J0^-1 = R
    sig, mu, prm = _mu_exp(G, J, np.linalg.inv(J0))
    rho, e, gam = 1.3, 2.0, 1.4
    ep = 0.5 * (e + math.sqrt(e * e + 1e-12))
    cs = math.sqrt(gam * (gam - 1) * ep)
    l0 = prm.l0_exp
    assert abs(l0 - 0.05) < 1e-15
    ref_mu = rho * (2.0 * l0 ** 2 * 0.7 + 0.5 * l0 * cs)
    assert abs(mu - ref_mu) <= 1e-14 * ref_mu
    assert np.abs(sig - (-(gam - 1) * rho * ep * np.eye(d) + ref_mu * G)).max() <= 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_mu_exp_directional_length(d):
    """A stretch a along x (J J0^-1 = diag(a, 1, ..)): compression along x sees l = a l0,
    compression along y sees l = l0; expansion only (lambda_1 > 0) drops the c_s term."""
    a = 2.5
    J0 = np.eye(d) * 0.25
    S = np.eye(d)
    S[0, 0] = a
    J = S @ J0
    Jinv0 = np.linalg.inv(J0)
    l0 = _prm(d).l0_exp
    for axis, ell in ((0, a * l0), (1, l0)):
        lam = np.full(d, 0.3)
        lam[axis] = -0.9
        _, mu, _ = _mu_exp(np.diag(lam), J, Jinv0, rho=1.0, e=0.0)
        cs = math.sqrt(1.4 * 0.4 * 0.5e-6)
        assert abs(mu - (2.0 * ell ** 2 * 0.9 + 0.5 * ell * cs)) <= 1e-14 * mu
    _, mu, _ = _mu_exp(np.diag(np.linspace(0.2, 0.6, d)), J, Jinv0, rho=1.0, e=1.0)
    assert abs(mu - 2.0 * (a * l0) ** 2 * 0.2) <= 1e-14 * mu        # smallest eigenvalue along x


def test_mu_exp_vorticity_switch():
    """psi_0 = |div v| / (sqrt(d) |grad v|_F): 1 for isotropic compression, 0 for a
    divergence-free flow (the q1 term vanishes), when the switch is on."""
    d = 2
    J0 = np.eye(d) * 0.25
    Jinv0 = np.linalg.inv(J0)
    l0 = _prm(d).l0_exp
    _, mu_on, _ = _mu_exp(-0.4 * np.eye(d), J0, Jinv0, rho=1.0, e=1.0, vorticity=True)
    _, mu_off, _ = _mu_exp(-0.4 * np.eye(d), J0, Jinv0, rho=1.0, e=1.0, vorticity=False)
    assert abs(mu_on - mu_off) <= 1e-15 * mu_off
    shear = np.array([[0.5, 0.3], [-0.1, -0.5]])          # trace-free, lambda_1 < 0
    _, mu_sw, _ = _mu_exp(shear, J0, Jinv0, rho=1.0, e=1.0, vorticity=True)
    lam1 = np.linalg.eigvalsh(0.5 * (shear + shear.T))[0]
    assert abs(mu_sw - 2.0 * l0 ** 2 * abs(lam1)) <= 1e-14 * mu_sw
