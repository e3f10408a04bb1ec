"""Pins of the oracle's SDIRK schemes (Sec. 4: SD2 = implicit midpoint, SD3 and SD4 the
3-stage methods of orders 3 and 4).

The tableaux are checked against the Runge-Kutta order conditions and the stability
properties that define them, the stage loop against the fully coupled stage system of a
linear ODE, and the whole step on the hydrodynamics residual by its temporal order."""
import numpy as np
import pytest

from oracle import problems, solver

# (order, rooted-tree condition) pairs: b^T Phi = 1 / gamma(tree) up to order 4
def _conditions(A, b):
    c = A.sum(axis=1)
    Ac = A @ c
    return [
        (1, b.sum(), 1.0),
        (2, b @ c, 1.0 / 2),
        (3, b @ (c * c), 1.0 / 3),
        (3, b @ Ac, 1.0 / 6),
        (4, b @ (c ** 3), 1.0 / 4),
        (4, b @ (c * Ac), 1.0 / 8),
        (4, b @ (A @ (c * c)), 1.0 / 12),
        (4, b @ (A @ Ac), 1.0 / 24),
    ]


def _stability(A, b, z):
    """R(z) = 1 + z b^T (I - z A)^-1 1 (the step's factor on y' = lambda y, z = lambda dt)."""
    s = len(b)
    return 1.0 + z * (b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s)))


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_tableau_order_conditions(scheme):
    A, b = solver.sdirk_tableau(scheme)
    assert np.allclose(np.triu(A, 1), 0.0)                  # diagonally implicit
    assert np.allclose(np.diag(A), A[0, 0])                 # singly diagonal
    for order, val, want in _conditions(A, b):
        if order <= scheme:
            assert abs(val - want) < 1e-14, (order, val, want)
    if scheme < 4:   # exactly of the stated order: some condition of the next order fails
        nxt = [abs(v - w) for o, v, w in _conditions(A, b) if o == scheme + 1]
        assert max(nxt) > 1e-3


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_a_stability(scheme):
    """All three are A-stable: |R(iy)| <= 1 on the imaginary axis with the poles 1/gamma in
    the right half-plane, so |R| <= 1 on the left half-plane (maximum principle)."""
    A, b = solver.sdirk_tableau(scheme)
    assert A[0, 0] > 0
    for y in np.concatenate([np.linspace(0.0, 50.0, 501), np.logspace(2, 8, 25)]):
        assert abs(_stability(A, b, 1j * y)) <= 1.0 + 1e-12
    for x in -np.logspace(-3, 6, 40):
        assert abs(_stability(A, b, x)) <= 1.0 + 1e-12


def test_sd3_is_l_stable_and_stiffly_accurate():
    A, b = solver.sdirk_tableau(3)
    assert np.array_equal(A[-1], b)                    # u^{n+1} is the last stage's state
    assert abs(_stability(A, b, -1e9)) < 1e-8          # R(-inf) = 0
    assert abs(_stability(*solver.sdirk_tableau(2), -1e9) + 1.0) < 1e-8   # midpoint: R(-inf) = -1


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_local_error_order(scheme):
    """|R(z) - e^z| = O(z^{p+1}): halving z divides it by about 2^{p+1}."""
    A, b = solver.sdirk_tableau(scheme)
    errs = [abs(_stability(A, b, z) - np.exp(z)) for z in (-0.04, -0.02)]
    assert 0.8 * 2 ** (scheme + 1) < errs[0] / errs[1] < 1.25 * 2 ** (scheme + 1)


@pytest.mark.parametrize("scheme", [2, 3, 4])
def test_stage_loop_matches_coupled_system(scheme):
    """On y' = L y the stage loop (one solve per stage, bases from earlier stages) must equal
    the coupled Runge-Kutta system (I - dt A (x) L) K = 1 (x) L y0, y1 = y0 + dt (b^T (x) I) K."""
    rng = np.random.default_rng(5)
    L = rng.standard_normal((5, 5)) - 3.0 * np.eye(5)
    y0 = rng.standard_normal(5)
    dt = 0.3
    A, b = solver.sdirk_tableau(scheme)
    s = len(b)

    def stage_solve(base, tau, guess):
        return np.linalg.solve(np.eye(5) - tau * L, L @ base)
    y1, ks = solver.sdirk_stages(stage_solve, y0, dt, A, b)
    K = np.linalg.solve(np.eye(5 * s) - dt * np.kron(A, L), np.tile(L @ y0, s))
    assert np.allclose(np.concatenate(ks), K, rtol=1e-12, atol=1e-12)
    assert np.allclose(y1, y0 + dt * np.kron(b, np.eye(5)) @ K, rtol=1e-12, atol=1e-12)


def test_sd2_step_is_the_implicit_midpoint_step():
    hyd, u = problems.taylor_green(2, 2, p0=100.0)
    ua, ka, _ = solver.implicit_midpoint_step(hyd, u, 0.003)
    ub, kb, res = solver.sdirk_step(hyd, u, 0.003, 2)
    assert len(res) == 1
    assert np.array_equal(ua, ub) and np.array_equal(ka, kb)


@pytest.mark.parametrize("scheme,lo,hi", [(2, 3.5, 4.6), (3, 7.0, 9.0), (4, 14.0, 28.0)])
def test_sdirk_temporal_order_on_taylor_green(scheme, lo, hi):
    """Q1-Q0 Taylor-Green on 2 x 2 elements to t = 0.004: halving dt divides the difference
    to a 32-step solution by about 2^p (p = 2, 3, 4)."""
    def run(nsteps):
        hyd, u = problems.taylor_green(2, 1, p0=100.0)
        kp = None
        for _ in range(nsteps):
            u, kp, _ = solver.sdirk_step(hyd, u, 0.004 / nsteps, scheme, kp, rtol=1e-13, atol=1e-13)
        return u
    ref = run(32)
    e = [np.linalg.norm(run(n) - ref) for n in (2, 4)]
    assert lo < e[0] / e[1] < hi, e
