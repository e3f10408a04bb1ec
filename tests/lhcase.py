"""Shared set-up for GPU parity tests: the same seeded state on the oracle and the GPU."""
import numpy as np
import torch

import lh_synth
from oracle import problems
from oracle.fem import Mesh as OMesh
from oracle.hydro import Hydro, Params


class Case:
    def __init__(self, dim, n, k, seed=0, visc=True, tg=False, lo=None, hi=None, rho0=1.0, gamma=1.4,
                 h_coarse=0.0, vscale=1.0, e_lo=0.0, visc_model='imp'):
        import paper_2609_16424_b300 as lh
        lo = lo or (0.0,) * dim
        hi = hi or (1.0,) * dim
        self.dim, self.n, self.k = dim, tuple(n), k
        m = OMesh(n, lo, hi, k)
        prm = Params(m, rho0=rho0, gamma=gamma, visc=visc, tg_source=tg, h_coarse=h_coarse or None,
                     visc_model=visc_model)
        self.hyd = Hydro(m, prm)
        self.u = problems.perturbed_state(self.hyd, lh_synth.perturbed_draws(n, k, seed, e_lo=e_lo),
                                         vscale=vscale)
        self.gm = lh.Mesh(dim, n, lo, hi, k, rho0=rho0, gamma=gamma, visc=visc, tg_source=tg,
                          h_coarse=h_coarse)
        assert self.gm.n == m.n_unknowns and self.gm.NV == m.NV and self.gm.NEd == m.NEd
        self.nx = dim * m.NV

    def dev(self, a, dtype=torch.float64):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")

    def blocks(self, a):
        a = np.asarray(a)
        return a[:self.nx], a[self.nx:2 * self.nx], a[2 * self.nx:]

    def rel_blocks(self, got, ref):
        out = []
        for g, r in zip(self.blocks(got), self.blocks(ref)):
            den = np.linalg.norm(r)
            out.append(np.linalg.norm(g - r) / (den if den > 0 else 1.0))
        return out
