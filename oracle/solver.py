"""Inexact Newton with backtracking line search and the implicit midpoint step.

Sec. 3.5: solve R(k; tau, u) = 0 (Eq. (21)) by Newton, J(k^m) dk^m = -r^m (Eq. (22)),
with a backtracking line search that rejects trial updates producing a non-positive
Jacobian determinant at any quadrature point.  Sec. 4.1: the order-2 SDIRK method is
the implicit midpoint rule (one stage, tau = dt / 2, u^{n+1} = u^n + dt k).

Readings where the paper is silent: stop when ||r||_2 <= rtol ||r^0||_2 (or below an
absolute floor); halve the step up to 10 times; initial guess k^0 = previous k (zero at
the first step).  The linear solve is exact (dense LU of the complex-step Jacobian) on
small systems and preconditioned GMRES with complex-step Jacobian actions otherwise;
the converged Newton solution does not depend on that choice.

Also the Newton-count time step control of Sec. 4 ("Implicit time step control") and the
three SDIRK schemes of Sec. 4 (SD2/SD3/SD4: implicit midpoint, and the 3-stage methods of
orders 3 and 4).  Each stage i solves the stage system of Eq. (21),
R(k_i; a_ii dt, u^n + dt sum_{j<i} a_ij k_j) = 0, and u^{n+1} = u^n + dt sum_i b_i k_i.
The paper names the schemes only by order and stage count; the tableaux are the classical
ones with those properties (reading): Alexander's L-stable stiffly accurate method (gamma the
root in (1/6, 1/2) of gamma^3 - 3 gamma^2 + 3/2 gamma - 1/6) and Crouzeix's A-stable method
(gamma = 1/2 + cos(pi/18)/sqrt(3)).  Stage initial guesses: the previous stage's k (the
caller's k_prev, or zero, for the first stage).
"""
import numpy as np


class NewtonResult:
    def __init__(self):
        self.iters = 0
        self.backtracks = 0
        self.r0 = 0.0
        self.rfinal = 0.0
        self.converged = False
        self.lin_iters = 0


def _block_prec(hyd):
    """Block-diagonal preconditioner diag(I, M_V^-1, M_E^-1) (exact mass solves)."""
    import scipy.sparse.linalg as spla
    m = hyd.m
    Mv = hyd.mass_v_sparse().tocsc()
    lu = spla.splu(Mv)
    MeInv = np.linalg.inv(hyd.mass_e_elem())
    n1 = m.d * m.NV

    def apply(r):
        out = r.copy()
        rv = r[n1:2 * n1].reshape(m.d, m.NV)
        out[n1:2 * n1] = np.concatenate([lu.solve(rv[c]) for c in range(m.d)])
        re = r[2 * n1:].reshape(m.NE, m.NL)
        out[2 * n1:] = np.einsum('eab,eb->ea', MeInv, re).ravel()
        return out
    return apply


def newton(hyd, u, tau, k0=None, rtol=1e-10, atol=1e-14, maxit=20, lin='auto',
           lin_rtol=1e-12, max_halvings=10, lag=False):
    """Solve R(k; tau, u) = 0.  Returns (k, NewtonResult).

    lin: 'dense' (dense complex-step Jacobian + LU), 'sparse' (compressed complex-step
    Jacobian + sparse LU), 'gmres' (preconditioned GMRES on complex-step actions) or
    'auto' (dense up to 800 unknowns, sparse above).  lag=True keeps the first
    Jacobian of the solve for all its iterations (chord Newton).
    """
    n = u.size
    k = np.zeros(n) if k0 is None else k0.copy()
    res = NewtonResult()
    if lin == 'auto':
        lin = 'dense' if n <= 800 else 'sparse'
    prec = None
    lu = None
    pattern = colors = None
    for it in range(maxit + 1):
        r = hyd.residual(u, k, tau)
        nr = float(np.linalg.norm(r))
        if it == 0:
            res.r0 = nr
        res.rfinal = nr
        if nr <= max(rtol * res.r0, atol):
            res.converged = True
            break
        if it == maxit:
            break
        if lin == 'dense':
            dk = np.linalg.solve(hyd.jacobian(u, k, tau), -r)
        elif lin == 'sparse':
            import scipy.sparse.linalg as spla
            from .hydro import jacobian_sparse, coupling_pattern, column_colors
            if pattern is None:
                pattern, colors = coupling_pattern(hyd.m), column_colors(hyd.m)
            if lu is None or not lag:
                lu = spla.splu(jacobian_sparse(hyd, u, k, tau, pattern, colors))
            dk = lu.solve(-r)
        else:
            import scipy.sparse.linalg as spla
            if prec is None:
                prec = _block_prec(hyd)
            A = spla.LinearOperator((n, n), matvec=lambda z: hyd.jvp_complex_step(u, k, tau, z))
            Pm = spla.LinearOperator((n, n), matvec=prec)
            count = [0]

            def cb(_):
                count[0] += 1
            dk, _info = spla.gmres(A, -r, M=Pm, rtol=lin_rtol, atol=0.0, restart=100,
                                   maxiter=20, callback=cb, callback_type='pr_norm')
            res.lin_iters += count[0]
        lam = 1.0
        for _ in range(max_halvings + 1):
            kt = k + lam * dk
            wx = hyd.m.split(u + tau * kt)[0]
            if hyd.min_detj(wx) > 0.0:
                break
            lam *= 0.5
            res.backtracks += 1
        k = kt
        res.iters += 1
    return k, res


def implicit_midpoint_step(hyd, u, dt, k_prev=None, **kw):
    """One implicit midpoint step: tau = dt / 2, u^{n+1} = u^n + dt k."""
    k, res = newton(hyd, u, 0.5 * dt, k0=k_prev, **kw)
    return u + dt * k, k, res


def dt_control(dt, newton_iters):
    """Sec. 4 time step control: <= 1 iteration -> x1.05; 2-3 -> keep; >= 4 -> reject, x0.85.

    Returns (new_dt, accepted).
    """
    if newton_iters <= 1:
        return 1.05 * dt, True
    if newton_iters <= 3:
        return dt, True
    return 0.85 * dt, False


def sdirk_tableau(scheme):
    """Butcher tableau (A [s x s] lower triangular with equal diagonal, b [s]) of SD2/SD3/SD4."""
    if scheme == 2:
        return np.array([[0.5]]), np.array([1.0])
    if scheme == 3:
        r = np.roots([1.0, -3.0, 1.5, -1.0 / 6.0])
        g = float(min(r.real[(abs(r.imag) < 1e-12) & (r.real > 1.0 / 6.0) & (r.real < 0.5)]))
        b1 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0
        b2 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0
        A = np.array([[g, 0.0, 0.0], [(1.0 - g) / 2.0, g, 0.0], [b1, b2, g]])
        return A, A[2].copy()
    if scheme == 4:
        g = 0.5 + np.cos(np.pi / 18.0) / np.sqrt(3.0)
        d = 1.0 / (6.0 * (2.0 * g - 1.0) ** 2)
        A = np.array([[g, 0.0, 0.0], [0.5 - g, g, 0.0], [2.0 * g, 1.0 - 4.0 * g, g]])
        return A, np.array([d, 1.0 - 2.0 * d, d])
    raise ValueError("scheme must be 2, 3 or 4")


def sdirk_stages(stage_solve, u, dt, A, b, k0=None):
    """The SDIRK stage loop for any stage solver stage_solve(base, tau, k_guess) -> k.

    Returns (u^{n+1}, [k_1 .. k_s])."""
    ks = []
    guess = k0
    for i in range(len(b)):
        base = u.copy()
        for j in range(i):
            base = base + dt * A[i, j] * ks[j]
        k = stage_solve(base, dt * A[i, i], guess)
        ks.append(k)
        guess = k
    unew = u.copy()
    for i in range(len(b)):
        unew = unew + dt * b[i] * ks[i]
    return unew, ks


def sdirk_step(hyd, u, dt, scheme, k_prev=None, **kw):
    """One SDn step (n = scheme): Newton on each stage system.  Returns (u^{n+1}, k_s,
    [NewtonResult per stage]); raises RuntimeError if a stage does not converge."""
    A, b = sdirk_tableau(scheme)
    results = []

    def solve(base, tau, guess):
        k, res = newton(hyd, base, tau, k0=guess, **kw)
        if not res.converged:
            raise RuntimeError("SDIRK stage did not converge")
        results.append(res)
        return k
    unew, ks = sdirk_stages(solve, u, dt, A, b, k_prev)
    return unew, ks[-1], results


def velocity_block_diagonal(hyd, u, k, tau):
    """Diagonal of the velocity block dR_v/dk_v = M_V + tau dF.1/dv of the stage Jacobian
    (the block the paper's Eq. (23) preconditions; identity on fixed rows), [d * NV], read
    off the complex-step sparse Jacobian."""
    from .hydro import jacobian_sparse
    n1 = hyd.m.d * hyd.m.NV
    return jacobian_sparse(hyd, u, k, tau).diagonal()[n1:2 * n1].copy()
