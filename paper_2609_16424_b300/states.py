"""Initial states of the point-blast problem built on the GPU (problem set-up, not the
hot path): corner deposit of a given total internal energy, v = 0, undeformed mesh."""
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
