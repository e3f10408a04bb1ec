"""Diagonal of the velocity block M_V + tau dF/dv (the block of the paper's Eq. (23)) and
the Jacobi preconditioner built on it (precond kind 2), against the oracle."""
import numpy as np
import pytest
import torch

import lh_synth
from lhcase import Case
from oracle import solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n,k", [(2, (3, 3), 2), (2, (2, 2), 3), (3, (2, 2, 2), 1), (3, (2, 2, 2), 2)])
def test_jvv_diagonal_matches_oracle(dim, n, k):
    c = Case(dim, n, k, seed=7, vscale=2.0)
    kk = lh_synth.normal_vector(c.u.size, 3, 0.2)
    tau = 0.05
    ref = solver.velocity_block_diagonal(c.hyd, c.u, kk, tau)
    mass = solver.velocity_block_diagonal(c.hyd, c.u, kk, 0.0)
    got = c.gm.jvv_diagonal(c.dev(c.u), c.dev(kk), tau).cpu().numpy()
    visc = ref - mass
    assert np.abs(visc).max() > 1e-3 * np.abs(mass).max()      # the viscous part is exercised
    err = np.abs(got - ref).max()
    assert err <= 5e-4 * np.abs(visc).max() + 1e-12 * np.abs(ref).max(), (err, np.abs(visc).max())


def test_jvv_jacobi_newton_reaches_the_root():
    import paper_2609_16424_b300 as lh
    c = Case(3, (4, 4, 4), 2, seed=3, vscale=1.0)
    u = c.dev(c.u)
    outs = []
    for pc in ("kron", "jvv_diag"):
        ug, kg = u.clone(), torch.zeros_like(u)
        st = c.gm.newton_step(ug, kg, 0.01, newton_rtol=1e-11, gmres_rtol=1e-8, gmres_maxit=300, restart=40,
                              jvp_prec="fp32", precond=pc)
        outs.append((ug.cpu().numpy(), st))
    (a, sa), (b, sb) = outs
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(a), (sa, sb)
    with pytest.raises(lh.LHError) as ei:
        c.gm.newton_step(u.clone(), None, 0.01, precond="jvv_diag")   # FP64 J.w has no record
    assert ei.value.status == 1


def test_jvv_jacobi_at_large_tau():
    """Large steps: where tau dF/dv pulls a diagonal entry below half of diag(M_V) (or makes it
    negative) the preconditioner keeps 0.5 diag(M_V); lh_jvv_diagonal still returns the
    diagonal itself.  Newton with it reaches the same root as with the exact mass inverse."""
    c = Case(3, (4, 4, 4), 2, seed=5, vscale=3.0)
    u = c.dev(c.u)
    tau = 0.02
    kk = torch.zeros_like(u)
    d = c.gm.jvv_diagonal(u, kk, tau).cpu().numpy()
    dm = c.gm.jvv_diagonal(u, kk, 0.0).cpu().numpy()
    free = dm != 1.0
    assert np.abs(d[free] - dm[free]).max() > 0.05 * np.abs(dm[free]).max()   # viscous part exercised
    outs = []
    for pc in ("kron", "jvv_diag"):
        ug, kg = u.clone(), torch.zeros_like(u)
        st = c.gm.newton_step(ug, kg, 2 * tau, newton_rtol=1e-11, gmres_rtol=1e-8, gmres_maxit=400, restart=40,
                              jvp_prec="fp32", precond=pc)
        outs.append((ug.cpu().numpy(), st))
    (a, sa), (b, sb) = outs
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(a), (sa, sb)


@pytest.mark.parametrize("degree", [1, 3, 5])
def test_chebyshev_velocity_block_reaches_the_root(degree):
    """Preconditioner kind 3: a Chebyshev iteration on the velocity Schur block
    S = M_V + tau dF.1/dv + tau^2 dF.1/dx (applied by the record J.w), Jacobi-scaled by the
    clamped diagonal of M_V + tau dF/dv.  A fixed polynomial in S, so right-preconditioned
    GMRES stays exact: Newton reaches the root of the exact-mass-inverse run.  (Degree 2 is
    left out: on this viscous state its residual polynomial does not contract the lower
    spectrum and GMRES needs hundreds of iterations.)"""
    c = Case(3, (4, 4, 4), 2, seed=5, vscale=3.0)
    u = c.dev(c.u)
    ref = u.clone()
    c.gm.newton_step(ref, torch.zeros_like(u), 0.04, newton_rtol=1e-11, gmres_rtol=1e-8, gmres_maxit=400,
                     restart=40, jvp_prec="fp32", precond="kron")
    ug = u.clone()
    st = c.gm.newton_step(ug, torch.zeros_like(u), 0.04, newton_rtol=1e-11, gmres_rtol=1e-8, gmres_maxit=400,
                          restart=40, jvp_prec="fp32", precond="cheb", cheb_degree=degree)
    a, b = ref.cpu().numpy(), ug.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(a), st
