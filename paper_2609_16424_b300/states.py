"""Initial states of the test problems built on the GPU (problem set-up, not the hot path):
the point blast (corner deposit of a given total internal energy) and the three-state
interface problem (three regions of density, pressure and gamma), v = 0, undeformed mesh."""
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
