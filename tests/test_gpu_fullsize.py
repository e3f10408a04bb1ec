"""Parity at the full workload sizes, in the launch configuration the benchmark times.

- 3D point-blast mesh 24^3 Q2-Q1 (the benchmark's size): the oracle evaluates the whole
  residual and the complex-step J.w (seconds) and every output is compared.
- Three-state interface problem 56x24 Q3-Q2 with per-element rho0 / gamma.
- The record J.w of 64-point elements at sizes where its warps walk element lists.
- 48^3 meshes (throughput sweep sizes, too large for the dense oracle): properties that hold
  at any size, checked on the GPU outputs alone.
"""
import numpy as np
import pytest
import torch

import lh_synth
from lhcase import Case
from oracle import problems

pytestmark = pytest.mark.gpu


def test_blast24_residual_and_jvp_full_vector():
    c = Case(3, (24, 24, 24), 2, seed=61)
    kk = lh_synth.normal_vector(c.gm.n, 62, 0.05)
    dk = lh_synth.normal_vector(c.gm.n, 63)
    tau = 1e-3
    u, kd = c.dev(c.u), c.dev(kk)
    ref = c.hyd.residual(c.u, kk, tau)
    got = c.gm.residual(u, kd, tau).cpu().numpy()
    assert max(c.rel_blocks(got, ref)) <= 1e-12
    jref = c.hyd.jvp_complex_step(c.u, kk, tau, dk)
    jgot = c.gm.jvp(u, kd, tau, c.dev(dk)).cpu().numpy()
    assert max(c.rel_blocks(jgot, jref)) <= 1e-11
    c.gm.linearize(u, kd, tau)
    jf = c.gm.jvp(u, kd, tau, c.dev(dk, torch.float32), lin=True).double().cpu().numpy()
    jref32 = c.hyd.jvp_complex_step(c.u, kk, tau, dk.astype(np.float32).astype(np.float64))
    assert max(c.rel_blocks(jf, jref32)) <= 2e-5
    # tensor-core J.w (bounds: five unit roundoffs of TF32 / BF16; x rows stay FP32)
    for kind, tol in (("tf32", 5 * 2.0 ** -11), ("bf16", 5 * 2.0 ** -9)):
        jt = c.gm.jvp(u, kd, tau, c.dev(dk, torch.float32), tc=kind).double().cpu().numpy()
        rel = c.rel_blocks(jt, jref32)
        assert rel[0] <= 2e-5 and max(rel[1:]) <= tol, (kind, rel)
    c.gm.tc_status()


@pytest.mark.parametrize("dim,n,k", [(2, (56, 48), 4), (3, (17, 15, 11), 2)])
def test_record_jvp_element_lists(dim, n, k):
    """The record J.w for elements of 64 points (2D Q4, 3D Q2: one warp per element walking a
    strided element list, the next record arriving by bulk copy) at sizes with more elements
    than resident warps (2368 on a B300) and not a multiple of them: warps take one or two
    elements, each output is compared with the oracle's complex-step J.w."""
    c = Case(dim, n, k, seed=64)
    kk = lh_synth.normal_vector(c.gm.n, 65, 0.05)
    dk = lh_synth.normal_vector(c.gm.n, 66)
    tau = 1e-3
    u, kd = c.dev(c.u), c.dev(kk)
    c.gm.linearize(u, kd, tau)
    jf = c.gm.jvp(u, kd, tau, c.dev(dk, torch.float32), lin=True).double().cpu().numpy()
    jref = c.hyd.jvp_complex_step(c.u, kk, tau, dk.astype(np.float32).astype(np.float64))
    assert max(c.rel_blocks(jf, jref)) <= 2e-5


def test_interface_problem_full_size():
    """56x24 Q3-Q2 on [0,7]x[0,3], three regions (rho, p, gamma) by element centre."""
    import paper_2609_16424_b300 as lh
    hyd, u0 = problems.triple_point(56, 24, 3)
    gm = lh.Mesh(2, (56, 24), (0.0, 0.0), (7.0, 3.0), 3, rho0=hyd.p.rho0, gamma=hyd.p.gamma)
    m = hyd.m
    draws = lh_synth.perturbed_draws((56, 24), 3, 64)
    u = problems.perturbed_state(hyd, {"xi": draws["xi"], "v": draws["v"], "e": u0[2 * 2 * m.NV:]})
    kk = lh_synth.normal_vector(m.n_unknowns, 65, 0.05)
    tau = 2e-3
    ref = hyd.residual(u, kk, tau)
    ud, kd = torch.tensor(u, device="cuda"), torch.tensor(kk, device="cuda")
    got = gm.residual(ud, kd, tau).cpu().numpy()
    nx = 2 * m.NV
    for g, r in ((got[:nx], ref[:nx]), (got[nx:2 * nx], ref[nx:2 * nx]), (got[2 * nx:], ref[2 * nx:])):
        assert np.linalg.norm(g - r) <= 1e-12 * np.linalg.norm(r)
    dk = lh_synth.normal_vector(m.n_unknowns, 66)
    jref = hyd.jvp_complex_step(u, kk, tau, dk)
    jgot = gm.jvp(ud, kd, tau, torch.tensor(dk, device="cuda")).cpu().numpy()
    assert np.linalg.norm(jgot - jref) <= 1e-11 * np.linalg.norm(jref)
    # TF32 tensor-core J.w from the record (the interface workload's reduced-precision form)
    dk32 = dk.astype(np.float32).astype(np.float64)
    jref32 = hyd.jvp_complex_step(u, kk, tau, dk32)
    gm.linearize(ud, kd, tau)
    jt = gm.jvp(ud, kd, tau, torch.tensor(dk32, device="cuda", dtype=torch.float32), tc="tf32")
    jt = jt.double().cpu().numpy()
    assert np.linalg.norm(jt[:nx] - jref32[:nx]) <= 2e-5 * np.linalg.norm(jref32[:nx])
    for g, r in ((jt[nx:2 * nx], jref32[nx:2 * nx]), (jt[2 * nx:], jref32[2 * nx:])):
        assert np.linalg.norm(g - r) <= 5 * 2.0 ** -11 * np.linalg.norm(r)
    gm.tc_status()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sweep_size_properties(k):
    """48^3 Q_k - Q_{k-1}, no walls, k = 0, tau = 0: R_v = F.1 and R_e = -F^T v, so
    sum_nodes R_v = 0 per component (partition of unity) and v.R_v + sum R_e = 0 (the
    compatible pair of Eq. (7)); checked in double on the GPU outputs."""
    import paper_2609_16424_b300 as lh
    n = (48, 48, 48)
    gm = lh.Mesh(3, n, (0, 0, 0), (1, 1, 1), k, gamma=1.4, bc_mask=0)
    x0 = gm.initial_nodes()
    d = lh_synth.perturbed_draws(n, k, 70 + k)
    nv = gm.NV
    interior = torch.ones(nv, dtype=torch.bool, device="cuda")
    ids = torch.arange(nv, device="cuda")
    for c, ext in enumerate((k * 48 + 1,) * 3):
        coord = (ids // (ext ** c)) % ext
        interior &= (coord > 0) & (coord < ext - 1)
    xi = torch.tensor(d["xi"], device="cuda") * interior
    u = torch.zeros(gm.n, dtype=torch.float64, device="cuda")
    u[:3 * nv] = x0 + (0.1 / 48 / k) * xi.reshape(-1)
    u[3 * nv:6 * nv] = torch.tensor(d["v"], device="cuda").reshape(-1)
    u[6 * nv:] = torch.tensor(d["e"], device="cuda")
    r = gm.residual(u, torch.zeros_like(u), 0.0)
    rv = r[3 * nv:6 * nv].reshape(3, nv)
    scale = rv.abs().sum(dim=1)
    assert torch.all(rv.sum(dim=1).abs() <= 1e-11 * scale)
    work = (u[3 * nv:6 * nv] * r[3 * nv:6 * nv]).sum() + r[6 * nv:].sum()
    assert abs(work.item()) <= 1e-11 * (u[3 * nv:6 * nv].abs() * r[3 * nv:6 * nv].abs()).sum().item()
