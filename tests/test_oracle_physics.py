"""Pins of the oracle's quadrature-point stress and discrete operators.

Each check is a value or an identity that the paper or the mathematics fixes, not a
re-typing of the oracle's formulas.
"""
import numpy as np
import pytest

import lh_synth
from oracle import problems
from oracle.fem import Mesh
from oracle.hydro import Hydro, Params, stress, det


def _prm(d, psi0=0.5, visc=True):
    m = Mesh((1,) * d, (0.0,) * d, (1.0,) * d, 1)
    prm = Params(m, visc=visc, psi0=psi0, h0=0.1, h_coarse=0.2)
    prm.detJ0 = np.array(1.0)
    return prm


def _mu_p(grad_v, e, rho, gamma, prm, d):
    """Viscosity coefficient and pressure recovered from a stress with zero-trace shear."""
    sig = stress(grad_v, np.array(1.0), np.array(rho), np.array(e), np.array(gamma), prm, d)
    return sig


def test_energy_regularisation_values():
    """Eq. (19)-(20): e = 0 gives e+ = eps_e / 2 and finite c_s; e >> eps_e gives p = (g-1) rho e."""
    prm = _prm(2, visc=False)
    z = np.zeros((2, 2))
    s0 = stress(z, np.array(1.0), np.array(2.0), np.array(0.0), np.array(1.4), prm, 2)
    assert abs(-s0[0, 0] / (0.4 * 2.0 * 0.5e-6) - 1) < 1e-12
    s1 = stress(z, np.array(1.0), np.array(2.0), np.array(3.0), np.array(1.4), prm, 2)
    assert abs(-s1[0, 0] - 0.4 * 2.0 * 3.0) < 1e-12
    assert s1[0, 1] == 0.0


def _e_plus(e, eps=1e-6):
    """e+ recovered from the pressure of a viscosity-free stress: p = (gamma - 1) rho e+."""
    prm = _prm(2, visc=False)
    prm.eps_e = eps
    z = np.zeros((2, 2))
    rho, gam = 1.7, 1.4
    sig = stress(z, np.array(1.0), np.array(rho), np.array(float(e)), np.array(gam), prm, 2)
    return -sig[0, 0] / ((gam - 1.0) * rho)


@pytest.mark.parametrize("e", [-1e-7, -1e-6, -1.0, -100.0, -1e8, 3e-7])
def test_energy_regularisation_negative_branch(e):
    """Eq. (19) for e < 0 as well as e > 0.  e+ = (e + sqrt(e^2 + eps^2)) / 2 is the larger
    root of x^2 - e x - eps^2/4 = 0, so e+ (e+ - e) = eps^2 / 4 and e+ > max(e, 0) at every
    e; dropping the factor 1/2 in either evaluation branch breaks the product by a factor
    2 or 4.  Checked to a few ulps of the product (for e >> eps the difference e+ - e
    cancels, so the positive side is checked at e ~ eps here and by its limit below)."""
    eps = 1e-6
    ep = _e_plus(e, eps)
    assert ep > 0.0 and ep > e
    assert abs(ep * (ep - e) / (0.25 * eps * eps) - 1.0) < 1e-12, (e, ep)


def test_energy_regularisation_negative_limits():
    """Eq. (19): e+ is increasing in e, continuous through e = 0 (value eps/2), and behaves
    like eps^2 / (4 |e|) as e -> -infinity (and like e as e -> +infinity)."""
    eps = 1e-6
    es = np.concatenate([-np.logspace(8, -12, 81), [0.0], np.logspace(-12, 8, 81)])
    ep = np.array([_e_plus(e, eps) for e in es])
    assert np.all(np.diff(ep) > 0)
    assert abs(_e_plus(-1e-15, eps) / (0.5 * eps) - 1) < 1e-8
    assert abs(_e_plus(1e-15, eps) / (0.5 * eps) - 1) < 1e-8
    for e in (-1e3, -1e6, -1e8):
        assert abs(_e_plus(e, eps) * 4.0 * abs(e) / eps ** 2 - 1.0) < 1e-9
    assert abs(_e_plus(1e6, eps) / 1e6 - 1.0) < 1e-15


@pytest.mark.parametrize("psi0", [0.3, 0.5, 0.7])
def test_switch_value_at_zero_compression(psi0):
    """Eq. (17): the shift makes psi(0) = psi0; Eq. (16): |0|_ds = ds; so at div v = 0,
    mu = rho h (q2 ds + q1 c_s psi0) with ds = 2 (h / h_coarse) c_s (Eq. (18))."""
    prm = _prm(2, psi0=psi0)
    shear = 0.8
    g = np.array([[0.0, shear], [0.0, 0.0]])        # trace-free
    rho, e, gam = 1.3, 2.0, 1.4
    sig = stress(g, np.array(1.0), np.array(rho), np.array(e), np.array(gam), prm, 2)
    mu = sig[0, 1] / (0.5 * shear)
    ep = 0.5 * (e + np.sqrt(e * e + 1e-12))
    cs = np.sqrt(gam * (gam - 1) * ep)
    h = prm.h0
    ds = 2 * h / prm.h_coarse * cs
    assert abs(mu - rho * h * (prm.q2 * ds + prm.q1 * cs * psi0)) < 1e-12 * mu


def test_switch_limits():
    """Strong compression: psi -> 1 and |dv|_ds -> |dv|; strong expansion: psi -> 0."""
    prm = _prm(2)
    rho, e, gam = 1.0, 1.0, 1.4
    cs = np.sqrt(gam * (gam - 1) * e)
    h = prm.h0
    for div, q1_on in [(-2e4, 1.0), (2e4, 0.0)]:
        g = np.diag([div / 2, div / 2])
        sig = stress(g, np.array(1.0), np.array(rho), np.array(e), np.array(gam), prm, 2)
        p = (gam - 1) * rho * e
        mu = (sig[0, 0] + p) / (div / 2)
        expect = rho * h * (prm.q2 * abs(h * div) + q1_on * prm.q1 * cs)
        assert abs(mu / expect - 1) < 1e-6


def test_mass_matrices():
    hyd, u = problems.sedov(3, 2, 2)
    Mv = hyd.mass_v_dense()
    total = hyd.total_mass()
    assert abs(total - 1.0) < 1e-14
    assert abs(Mv.sum() - total) < 1e-13
    assert np.allclose(Mv, Mv.T) and np.linalg.eigvalsh(Mv).min() > 0
    f = np.random.default_rng(0).normal(size=(2, hyd.m.NV))
    assert np.allclose(hyd.apply_mass_v(f), f @ Mv.T, atol=1e-14)
    Me = hyd.mass_e_elem()
    assert abs(Me.sum() - total) < 1e-13
    assert np.all(np.linalg.eigvalsh(Me).min(axis=1) > 0)


def _state(n, k, seed, visc=True, d=2):
    m = Mesh((n,) * d, (0.0,) * d, (1.0,) * d, k)
    prm = Params(m, gamma=1.4, visc=visc)
    hyd = Hydro(m, prm)
    u = problems.perturbed_state(hyd, lh_synth.perturbed_draws((n,) * d, k, seed))
    return hyd, u


@pytest.mark.parametrize("d,k", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_pressure_force_is_a_gradient(d, k):
    """Without viscosity alpha detJ p = (g-1) m_q e+ does not depend on x, so
    F.1 = -grad_x Phi with Phi(x) = sum_q (g-1) m_q e+_q ln det J_q(x) (Eq. (7))."""
    hyd, u = _state(2, k, 1, visc=False, d=d)
    m = hyd.m
    x, v, e = m.split(u)
    F, _ = hyd.force_matrix(x, v, e)
    F1 = m.scatter(F.sum(axis=3))
    eq = np.einsum('ej,qj->eq', e, m.Bl)
    ep = 0.5 * (eq + np.sqrt(eq ** 2 + 1e-12))
    coef = (hyd.p.gamma[:, None] - 1) * hyd.mq * ep

    def phi(xx):
        return np.sum(coef * np.log(det(np.einsum('ecn,qrn->eqcr', m.gather(xx), m.Gh))))
    g = np.zeros_like(x)
    hstep = 1e-6
    for c in range(d):
        for i in range(m.NV):
            xp, xm = x.copy(), x.copy()
            xp[c, i] += hstep
            xm[c, i] -= hstep
            g[c, i] = (phi(xp) - phi(xm)) / (2 * hstep)
    assert np.allclose(F1, -g, atol=1e-6 * np.abs(g).max())


@pytest.mark.parametrize("d,k", [(2, 2), (3, 1), (3, 2)])
def test_momentum_and_invariances(d, k):
    hyd, u = _state(2, k, 2, visc=True, d=d)
    m = hyd.m
    x, v, e = m.split(u)
    F, _ = hyd.force_matrix(x, v, e)
    F1 = m.scatter(F.sum(axis=3))
    # partition of unity of the H1 basis: total force vanishes (momentum conservation)
    assert np.all(np.abs(F1.sum(axis=1)) < 1e-12 * np.abs(F1).max())
    # translation of x and a uniform added velocity leave F unchanged
    Ft, _ = hyd.force_matrix(x + 0.37, v + 0.21, e)
    assert np.allclose(Ft, F, atol=1e-12 * np.abs(F).max())
    # a rigid rotation of x and v rotates the force rows
    rng = np.random.default_rng(3)
    Rm, _ = np.linalg.qr(rng.normal(size=(d, d)))
    if np.linalg.det(Rm) < 0:
        Rm[:, 0] *= -1
    Fr, _ = hyd.force_matrix(Rm @ x, Rm @ v, e)
    assert np.allclose(Fr, np.einsum('cb,ebnj->ecnj', Rm, F), atol=1e-11 * np.abs(F).max())


def test_uniform_compression_closed_form():
    """Affine box, v = -c (x - x_c): grad v = -c I at every point, so sigma is the
    isotropic -(p + c mu) I and F.1 = -(p + c mu) dVol/dx with dVol/dx from the
    outward face normals (boundary nodes only)."""
    m = Mesh((1, 1), (0.0, 0.0), (1.0, 1.0), 1)
    prm = Params(m, gamma=1.4, visc=True, h0=1.0, h_coarse=1.0)
    hyd = Hydro(m, prm)
    c = 0.3
    x0 = hyd.x0
    v = -c * (x0 - 0.5)
    e = np.full((1, 1), 2.0)
    F, _ = hyd.force_matrix(x0, v, e)
    F1 = m.scatter(F.sum(axis=3))
    # corners of the unit square: dArea/dx_i = 1/2 (y_{i+1} - y_{i-1}), counter-clockwise
    dA = np.array([[-0.5, 0.5, -0.5, 0.5], [-0.5, -0.5, 0.5, 0.5]])
    peff = -F1[0, 0] / dA[0, 0]
    assert np.allclose(F1, -peff * dA, atol=1e-14)
    ep = 0.5 * (2.0 + np.sqrt(4.0 + 1e-12))
    p = 0.4 * 1.0 * ep
    assert peff > p            # compression adds viscous pressure


def test_jacobian_structure_and_fd():
    """J = dR/dk: at tau = 0 it is diag(I, M_V (fixed rows: I), M_E); J_xv = -tau I;
    the complex-step J agrees with central differences."""
    hyd, u = _state(2, 2, 4, visc=True)
    m = hyd.m
    n = u.size
    k = lh_synth.normal_vector(n, 5, 0.1)
    J0 = hyd.jacobian(u, k, 0.0)
    n1 = m.d * m.NV
    Mv = hyd.mass_v_dense()
    Jvv = np.kron(np.eye(m.d), Mv)
    fixed = hyd.fixed.ravel()
    Jvv[fixed, :] = 0.0
    Jvv[fixed, fixed] = 1.0
    Me = hyd.mass_e_elem()
    expect = np.zeros((n, n))
    expect[:n1, :n1] = np.eye(n1)
    expect[n1:2 * n1, n1:2 * n1] = Jvv
    for e_ in range(m.NE):
        s = 2 * n1 + e_ * m.NL
        expect[s:s + m.NL, s:s + m.NL] = Me[e_]
    assert np.allclose(J0, expect, atol=1e-14)
    tau = 0.02
    J = hyd.jacobian(u, k, tau)
    assert np.allclose(J[:n1, n1:2 * n1], -tau * np.eye(n1), atol=1e-15)
    dk = lh_synth.normal_vector(n, 6)
    a = J @ dk
    b = hyd.jvp_fd(u, k, tau, dk, 1e-6)
    assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(a)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_taylor_green_l1_error_of_the_interpolant(k):
    """The L1 velocity error (Sec. 4.1 table) of the nodal Q_k interpolant of the exact
    Taylor-Green velocity falls as h^(k+1); the pressure level p0 does not enter it."""
    errs = [problems.l1_velocity_error(*problems.taylor_green(n, k)) for n in (4, 8)]
    assert abs(np.log2(errs[0] / errs[1]) - (k + 1)) < 0.1, errs
    hyd, u = problems.taylor_green(4, k, p0=100.0)
    assert problems.l1_velocity_error(hyd, u) == errs[0]
