"""Initial states of the paper's test problems, built from their definitions.

* Taylor-Green vortex (Sec. 4.1): rho = 1, v = (sin pi x cos pi y, -cos pi x sin pi y),
  p = p0 + (cos 2 pi x + cos 2 pi y) / 4, gamma = 5/3, no viscosity, energy source on,
  walls (v.n = 0) on all sides.  The paper defers the set-up to its reference [Dobrev 2012,
  Sec. 8.1] and prints no p0; p0 = 1 (sound speed about 1.3) is the reading that fits the
  step counts of its Taylor-Green table (35 explicit steps at h = 1/16, CFL 0.5), p0 = 100
  a stiffer low-Mach variant that several tests use.  e = p / ((gamma - 1) rho) at the L2 nodes, v at the
  H1 nodes (nodal interpolation).
* Sedov point blast (Sec. 4.2): rho = 1, v = 0, gamma = 1.4, total internal energy
  0.25 deposited in the element at the origin, e = 0 elsewhere, walls on all sides.
* Three-state interface problem (Sec. 4.3): three regions of given rho, p, gamma,
  v = 0, walls on all sides; region by element centre.
* Synthetic perturbed state: interior nodes displaced, random v and e, from the
  seeded draws of ``lh_synth`` (the draws are inputs; their use is here).
"""
import numpy as np

from .fem import Mesh
from .hydro import Hydro, Params


def taylor_green(n=8, k=2, p0=1.0):
    """p = p0 + (cos 2 pi x + cos 2 pi y) / 4; the energy source does not depend on p0."""
    m = Mesh((n, n), (0.0, 0.0), (1.0, 1.0), k)
    prm = Params(m, rho0=1.0, gamma=5.0 / 3.0, visc=False, tg_source=True)
    hyd = Hydro(m, prm)
    x0 = hyd.x0
    v = np.stack([np.sin(np.pi * x0[0]) * np.cos(np.pi * x0[1]),
                  -np.cos(np.pi * x0[0]) * np.sin(np.pi * x0[1])])
    pl = m.l2_node_positions()
    p = p0 + (np.cos(2 * np.pi * pl[:, 0]) + np.cos(2 * np.pi * pl[:, 1])) / 4.0
    e = p / ((5.0 / 3.0 - 1.0) * 1.0)
    return hyd, m.join(x0, v, e)


def tg_velocity(x):
    """Exact Taylor-Green velocity at physical points x [..., 2]."""
    return np.stack([np.sin(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1]),
                     -np.cos(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1])], axis=-1)


def l1_velocity_error(hyd, u):
    """sum_q alpha detJ |v_h(x_q) - v_exact(x_q)|_2 on the current mesh."""
    from .hydro import det
    m = hyd.m
    x, v, _ = m.split(u)
    xq = np.einsum('ecn,qn->eqc', m.gather(x), m.Bh)
    vq = np.einsum('ecn,qn->eqc', m.gather(v), m.Bh)
    detJ = det(np.einsum('ecn,qrn->eqcr', m.gather(x), m.Gh))
    err = np.linalg.norm(vq - tg_velocity(xq), axis=-1)
    return float(np.sum(m.alpha[None, :] * detJ * err))


def sedov(n=4, k=2, d=3, energy=0.25, h_coarse=None):
    m = Mesh((n,) * d, (0.0,) * d, (1.0,) * d, k)
    prm = Params(m, rho0=1.0, gamma=1.4, visc=True, h_coarse=h_coarse)
    hyd = Hydro(m, prm)
    e = np.zeros((m.NE, m.NL))
    vol0 = float(np.prod(m.h))
    e[0, :] = energy / (1.0 * vol0)          # element 0 touches the origin
    return hyd, m.join(hyd.x0, np.zeros((d, m.NV)), e)


def triple_point(nx=56, ny=24, k=3):
    m = Mesh((nx, ny), (0.0, 0.0), (7.0, 3.0), k)
    c = m.element_centres()
    left = c[:, 0] < 1.0
    top = (~left) & (c[:, 1] > 1.5)
    rho = np.where(left, 1.0, np.where(top, 0.125, 1.0))
    p = np.where(left, 1.0, 0.1)
    gam = np.where(left, 1.5, np.where(top, 1.5, 1.4))
    prm = Params(m, rho0=rho, gamma=gam, visc=True)
    hyd = Hydro(m, prm)
    e_el = p / ((gam - 1.0) * rho)
    e = np.repeat(e_el[:, None], m.NL, axis=1)
    return hyd, m.join(hyd.x0, np.zeros((2, m.NV)), e)


def perturbed_state(hyd, draws, disp=0.1, vscale=1.0):
    """State from seeded draws: interior nodes moved by disp*h/k*U(-1,1), v and e given.

    ``draws`` holds arrays 'xi' [d, NV] in [-1, 1], 'v' [d, NV] and 'e' [NE*NL] (see
    lh_synth.perturbed_draws).  Velocity components normal to fixed walls are zeroed.
    """
    m = hyd.m
    interior = ~m.boundary_mask((1 << (2 * m.d)) - 1).any(axis=0)
    x = hyd.x0 + disp * (m.h / m.k)[:, None] * draws['xi'] * interior[None, :]
    v = np.where(hyd.fixed, 0.0, vscale * draws['v'])
    return m.join(x, v, draws['e'])
