"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds only random draws and problem-size bookkeeping: no quadrature,
basis, geometry or physics.  Both the CUDA path and the oracle turn the same draws
into states with their own code.

Workload shapes follow the paper's test problems (Sec. 4): a 2D Taylor-Green vortex
on an 8x8 Q2-Q1 mesh, a 3D point blast on 24^3 Q2-Q1 hexes, a 2D three-state
interface problem on 56x24 Q3-Q2 quads and a 48^3 Q_k-Q_{k-1} throughput sweep.
"""
import numpy as np


def sizes(n, k):
    """(NE, NV, N_E, n_unknowns, NQ) for a box of n = (nx, ny[, nz]) elements, order k."""
    d = len(n)
    ne = int(np.prod(n))
    nv = int(np.prod([k * m + 1 for m in n]))
    n_e = ne * k ** d
    return ne, nv, n_e, 2 * d * nv + n_e, ne * (2 * k) ** d


def perturbed_draws(n, k, seed, v_sigma=0.1, e_lo=0.0, e_hi=1.0):
    """Draws for a perturbed state: 'xi' ~ U(-1,1) [d, NV], 'v' ~ N(0, v_sigma^2) [d, NV],
    'e' ~ U(e_lo, e_hi) [N_E]."""
    d = len(n)
    _, nv, n_e, _, _ = sizes(n, k)
    rng = np.random.default_rng(seed)
    return {
        'xi': rng.uniform(-1.0, 1.0, size=(d, nv)),
        'v': rng.normal(0.0, v_sigma, size=(d, nv)),
        'e': rng.uniform(e_lo, e_hi, size=n_e),
    }


def normal_vector(n_unknowns, seed, scale=1.0):
    """A direction dk ~ N(0, scale^2) of length n_unknowns."""
    return np.random.default_rng(seed).normal(0.0, scale, size=n_unknowns)


# Named workloads: (dimension-wise element counts, order k, box lo, box hi)
WORKLOADS = {
    'tg2d_8x8_q2q1': ((8, 8), 2, (0.0, 0.0), (1.0, 1.0)),
    'blast3d_24_q2q1': ((24, 24, 24), 2, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)),
    'interface2d_56x24_q3q2': ((56, 24), 3, (0.0, 0.0), (7.0, 3.0)),
    'blast3d_48_q1q0': ((48, 48, 48), 1, (0.0,) * 3, (1.0,) * 3),
    'blast3d_48_q2q1': ((48, 48, 48), 2, (0.0,) * 3, (1.0,) * 3),
    'blast3d_48_q3q2': ((48, 48, 48), 3, (0.0,) * 3, (1.0,) * 3),
    'blast3d_48_q4q3': ((48, 48, 48), 4, (0.0,) * 3, (1.0,) * 3),
}
