"""Initial states of the test problems built on the GPU (problem set-up, not the hot path):
the point blast (corner deposit of a given total internal energy), the three-state
interface problem (three regions of density, pressure and gamma), v = 0, and the 2D
Taylor-Green vortex; undeformed mesh."""
import math

import numpy as np
import torch


def blast_state(mesh, energy, rho0=1.0):
    """e = energy / (rho0 |K0|) in the element touching the origin, zero elsewhere."""
    x0 = mesh.initial_nodes()
    u = torch.zeros(mesh.n, dtype=torch.float64, device=mesh.device)
    nx = x0.numel()
    u[:nx] = x0
    vol0 = 1.0 / mesh.NE          # unit box
    nl = mesh.NEd // mesh.NE
    u[2 * nx:2 * nx + nl] = energy / (rho0 * vol0)
    return u


def interface_problem(nx=56, ny=24, k=3, device=None):
    """Three-state interface problem on [0,7]x[0,3] (Q_k-Q_{k-1}), regions by element centre:
    x < 1: rho 1, p 1, gamma 1.5; x > 1, y < 1.5: rho 1, p 0.1, gamma 1.4; x > 1, y > 1.5:
    rho 0.125, p 0.1, gamma 1.5; e = p / ((gamma - 1) rho) per element, v = 0.
    Returns (mesh, u)."""
    from .hydro import Mesh
    rho, gam, e_el = [], [], []
    for ey in range(ny):
        for ex in range(nx):
            cx, cy = (ex + 0.5) * 7.0 / nx, (ey + 0.5) * 3.0 / ny
            if cx < 1.0:
                r, p, g = 1.0, 1.0, 1.5
            elif cy > 1.5:
                r, p, g = 0.125, 0.1, 1.5
            else:
                r, p, g = 1.0, 0.1, 1.4
            rho.append(r)
            gam.append(g)
            e_el.append(p / ((g - 1.0) * r))
    mesh = Mesh(2, (nx, ny), (0.0, 0.0), (7.0, 3.0), k, rho0=rho, gamma=gam, device=device)
    x0 = mesh.initial_nodes()
    u = torch.zeros(mesh.n, dtype=torch.float64, device=mesh.device)
    u[:x0.numel()] = x0
    nl = mesh.NEd // mesh.NE
    u[2 * x0.numel():] = torch.tensor(e_el, dtype=torch.float64, device=mesh.device).repeat_interleave(nl)
    return mesh, u


def taylor_green_problem(n, k, p0=1.0, device=None):
    """2D Taylor-Green vortex (Sec. 4.1) on [0,1]^2 with n x n Q_k-Q_{k-1} elements: rho 1,
    gamma 5/3, no artificial viscosity, the energy source on, walls on all sides;
    v = (sin pi x cos pi y, -cos pi x sin pi y) at the H1 nodes and e = p / ((gamma - 1) rho)
    with p = p0 + (cos 2 pi x + cos 2 pi y) / 4 at the L2 nodes (the Gauss-Legendre points of
    each element).  The paper prints no p0; p0 = 1 fits the step counts of its Taylor-Green
    table, p0 = 100 is a stiffer low-Mach variant.  Returns (mesh, u)."""
    from .hydro import Mesh
    gamma = 5.0 / 3.0
    mesh = Mesh(2, (n, n), (0.0, 0.0), (1.0, 1.0), k, rho0=1.0, gamma=gamma, visc=False, tg_source=True,
                device=device)
    x0 = mesh.initial_nodes()
    nv = mesh.NV
    u = torch.zeros(mesh.n, dtype=torch.float64, device=mesh.device)
    u[:2 * nv] = x0
    x, y = x0[:nv], x0[nv:]
    u[2 * nv:3 * nv] = torch.sin(math.pi * x) * torch.cos(math.pi * y)
    u[3 * nv:4 * nv] = -torch.cos(math.pi * x) * torch.sin(math.pi * y)
    z = (np.polynomial.legendre.leggauss(k)[0] + 1.0) / 2.0        # L2 nodes on [0, 1]
    h = 1.0 / n
    e_idx = np.arange(n * n)
    ex, ey = e_idx % n, e_idx // n
    px = (ex[:, None, None] + z[None, None, :]) * h                 # [e][j1][j0]
    py = (ey[:, None, None] + z[None, :, None]) * h
    p = p0 + (np.cos(2 * math.pi * px) + np.cos(2 * math.pi * py)) / 4.0
    u[4 * nv:] = torch.tensor((p / (gamma - 1.0)).reshape(-1), dtype=torch.float64, device=mesh.device)
    return mesh, u
