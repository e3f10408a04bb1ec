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

Also the Newton-count time step control of Sec. 4 ("Implicit time step control").
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
