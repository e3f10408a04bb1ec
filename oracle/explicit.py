"""Explicit time integration of the semi-discrete system (the paper's comparison path).

Paper passages: Sec. 2.1, Eqs. (6a)-(6b): M_V dv/dt = -F.1, M_E de/dt = F^T v (+ the
manufactured source b when enabled), dx/dt = v; Sec. 2.2: in explicit runs F's
quadrature data are formed once per stage and applied twice (F.1 and F^T v), and the mass
matrices are inverted by CG; Sec. 4.1: the explicit integrators RK2 (the RK2-average scheme),
RK3 (strong-stability-preserving) and RK4 (classical), run at CFL 0.5 with the time step
control of the explicit method.

The paper defers the RK2-average scheme and the explicit step control to Dobrev et al.
2012 (Secs. 7.1 and 7.3), which it does not print.  Readings used here:

* RK2-average: with a(U) = -M_V^-1 F(U).1 (zero on fixed velocity rows) and
  g(U, w) = M_E^-1 (F(U)^T w + b(x)):
      v_h = v + dt/2 a(U),  e_h = e + dt/2 g(U, v_h),  x_h = x + dt/2 v_h,  U_h = (x_h, v_h, e_h)
      v_1 = v + dt a(U_h),  vbar = (v + v_1) / 2,
      e_1 = e + dt g(U_h, vbar),  x_1 = x + dt vbar.
  Total energy 1/2 v^T M_V v + 1^T M_E e changes by exactly dt 1^T b per step (zero
  without a source): the kinetic change is -dt vbar^T F(U_h).1 and the internal change
  +dt vbar^T F(U_h).1 + dt 1^T b.
* RK3 (Shu-Osher SSP) and RK4 (classical) on dU/dt = f(U) = (v, a(U), g(U, v)).
* Step control: dt_est(U) = CFL x min_q h_min,q / (c_s + mu / (rho h_min,q)) with
  h_min,q = sigma_min(J_q) / k (the estimate the implicit path's FS-CFL also multiplies);
  the first dt is dt_est(U^0); after a step, if dt_est(U^{n+1}) < dt the step is repeated
  with 0.85 dt, and if dt_est(U^{n+1}) > 1.25 dt the next dt is 1.02 dt.
"""
import numpy as np

from .hydro import det, stress, stress_exp


def _free_solver(hyd):
    """Sparse LU of M_V restricted to the free rows of each velocity component."""
    import scipy.sparse.linalg as spla
    m = hyd.m
    M = hyd.mass_v_sparse().tocsc()
    out = []
    for c in range(m.d):
        free = np.nonzero(~hyd.fixed[c])[0]
        lu = spla.splu(M[free][:, free].tocsc())
        out.append((free, lu))
    return out


class Explicit:
    """The explicit right-hand side pieces of Eqs. (6a)-(6b) on a Hydro operator set."""

    def __init__(self, hyd):
        self.hyd = hyd
        self.m = hyd.m
        self.lu_v = _free_solver(hyd)
        self.me_inv = np.linalg.inv(hyd.mass_e_elem())

    def assemble(self, u):
        """The force matrices F(U) of Eq. (7) (formed once per stage) and the source b(x)."""
        x, v, e = self.m.split(u)
        F, _ = self.hyd.force_matrix(x, v, e)
        b = self.hyd.source(x) if self.hyd.p.tg_source else None
        return F, b

    def f_one(self, Fb):
        """F.1 [d, NV] (the first application of F)."""
        return self.m.scatter(Fb[0].sum(axis=-1))

    def f_t(self, Fb, w):
        """F^T w + b [NE, NL] (the second application of F)."""
        out = np.einsum('ecnj,ecn->ej', Fb[0], self.m.gather(w))
        return out if Fb[1] is None else out + Fb[1]

    def accel(self, F1):
        """a = -M_V^-1 F.1 on free rows, 0 on fixed rows."""
        a = np.zeros_like(F1)
        for c, (free, lu) in enumerate(self.lu_v):
            a[c, free] = lu.solve(-F1[c, free])
        return a

    def edot(self, FTw):
        return np.einsum('eab,eb->ea', self.me_inv, FTw)

    def rhs(self, u):
        """f(U) = (v, a(U), g(U, v)) as one state-shaped vector."""
        m = self.m
        _, v, _ = m.split(u)
        Fb = self.assemble(u)
        return m.join(v, self.accel(self.f_one(Fb)), self.edot(self.f_t(Fb, v)))


def rk2_average_step(ex, u, dt):
    """One RK2-average step (reading in the module header)."""
    m = ex.m
    x, v, e = m.split(u)
    Fb = ex.assemble(u)
    vh = v + 0.5 * dt * ex.accel(ex.f_one(Fb))
    eh = e + 0.5 * dt * ex.edot(ex.f_t(Fb, vh))
    xh = x + 0.5 * dt * vh
    uh = m.join(xh, vh, eh)
    Fh = ex.assemble(uh)
    v1 = v + dt * ex.accel(ex.f_one(Fh))
    vbar = 0.5 * (v + v1)
    return m.join(x + dt * vbar, v1, e + dt * ex.edot(ex.f_t(Fh, vbar)))


# Butcher tableaux of the explicit Runge-Kutta methods named in Sec. 4.1
RK_TABLEAUX = {
    3: (np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.25, 0.25, 0.0]]), np.array([1 / 6, 1 / 6, 2 / 3])),
    4: (np.array([[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]]),
        np.array([1 / 6, 1 / 3, 1 / 3, 1 / 6])),
}


def rk_step(f, u, dt, A, b):
    """One explicit Runge-Kutta step of dU/dt = f(U) with the tableau (A, b)."""
    ks = []
    for i in range(len(b)):
        ui = u.copy()
        for j in range(i):
            if A[i, j] != 0.0:
                ui = ui + dt * A[i, j] * ks[j]
        ks.append(f(ui))
    out = u.copy()
    for i in range(len(b)):
        out = out + dt * b[i] * ks[i]
    return out


def explicit_step(ex, u, dt, scheme):
    """scheme 2: RK2-average, 3: RK3 SSP, 4: RK4."""
    if scheme == 2:
        return rk2_average_step(ex, u, dt)
    A, b = RK_TABLEAUX[scheme]
    return rk_step(ex.rhs, u, dt, A, b)


def dt_estimate(hyd, u):
    """min_q h_min,q / (c_s + mu / (rho h_min,q)), h_min,q = sigma_min(J_q) / k, with the
    viscosity of the operator set's model (mu = 0 without viscosity)."""
    m = hyd.m
    x, v, e = m.split(u)
    J, detJ, gradw, grad_v, eq, rho = hyd.qp_state(x, v, e)
    gam = hyd.p.gamma[:, None]
    root = np.sqrt(eq * eq + hyd.p.eps_e ** 2)
    e_plus = np.where(eq < 0, 0.5 * hyd.p.eps_e ** 2 / np.where(eq < 0, root - eq, 1.0), 0.5 * (eq + root))
    cs = np.sqrt(gam * (gam - 1.0) * e_plus)
    hmin = np.linalg.svd(J, compute_uv=False)[..., -1] / m.k
    if hyd.p.visc_model == 'exp':
        _, mu = stress_exp(grad_v, J, hyd.J0inv, rho, eq, gam, hyd.p, m.d, return_mu=True)
    else:
        _, mu = stress(grad_v, detJ, rho, eq, gam, hyd.p, m.d, return_mu=True)
    return float(np.min(hmin / (cs + mu / (rho * hmin))))


def explicit_advance(hyd, u, t_end, cfl, scheme, max_steps=100000):
    """Explicit run from t = 0 to t_end with the step control of the module header.
    Returns (u, steps, rejected)."""
    ex = Explicit(hyd)
    dt = cfl * dt_estimate(hyd, u)
    t, steps, rejected = 0.0, 0, 0
    while t < t_end - 1e-14 * max(1.0, t_end) and steps < max_steps:
        h = min(dt, t_end - t)
        un = explicit_step(ex, u, h, scheme)
        est = cfl * dt_estimate(hyd, un)
        if est < h:
            dt = 0.85 * dt
            rejected += 1
            continue
        u = un
        t += h
        steps += 1
        if est > 1.25 * dt:
            dt = 1.02 * dt
    return u, steps, rejected


def total_energy(hyd, u):
    return hyd.kinetic_energy(u) + hyd.internal_energy(u)


def detj_min(hyd, u):
    m = hyd.m
    x = m.split(u)[0]
    return float(np.min(det(np.einsum('ecn,qrn->eqcr', m.gather(x), m.Gh))))
