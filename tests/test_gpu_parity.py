"""GPU parity against the oracle: residual, Jacobian actions, mass operators.

Sizes span several thread blocks with a ragged last block (elements per block: 32 for
2D Q1, 8 for 2D Q2, 2 for 3D Q2, 1 for 3D Q3/Q4).  Tolerances: FP64 residual and
FP64 J.w relative L2 <= 1e-12 / 1e-11 per block (x, v, e rows) against the oracle's
residual and its complex-step derivative; FP32 J.w <= 2e-5.
"""
import numpy as np
import pytest
import torch

import lh_synth
from lhcase import Case

pytestmark = pytest.mark.gpu

CASES = [
    (2, (7, 5), 1, True, False),
    (2, (7, 5), 2, True, False),
    (2, (5, 3), 2, False, True),      # Taylor-Green source, no viscosity
    (2, (4, 3), 3, True, False),
    (2, (3, 2), 4, True, False),
    (3, (5, 4, 3), 1, True, False),
    (3, (3, 3, 3), 2, True, False),
    (3, (2, 2, 1), 3, True, False),
    (3, (1, 1, 2), 4, True, False),
]
IDS = [f"d{c[0]}_n{'x'.join(map(str, c[1]))}_k{c[2]}{'_visc' if c[3] else ''}{'_tg' if c[4] else ''}" for c in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request):
    dim, n, k, visc, tg = request.param
    return Case(dim, n, k, seed=11, visc=visc, tg=tg)


def test_initial_nodes(case):
    x0 = case.gm.initial_nodes().cpu().numpy()
    assert np.abs(x0 - case.hyd.x0.ravel()).max() <= 1e-14


def test_residual_parity(case):
    kk = lh_synth.normal_vector(case.gm.n, 3, 0.1)
    tau = 0.01
    ref, detj = case.hyd.residual(case.u, kk, tau, return_detj=True)
    got, md = case.gm.residual(case.dev(case.u), case.dev(kk), tau, min_detj=True)
    rel = case.rel_blocks(got.cpu().numpy(), ref)
    assert max(rel) <= 1e-12, rel
    assert abs(md - detj.min()) <= 1e-13 * abs(detj.min())


def test_jvp_fp64_parity(case):
    kk = lh_synth.normal_vector(case.gm.n, 4, 0.1)
    dk = lh_synth.normal_vector(case.gm.n, 5)
    tau = 0.02
    ref = case.hyd.jvp_complex_step(case.u, kk, tau, dk)
    got = case.gm.jvp(case.dev(case.u), case.dev(kk), tau, case.dev(dk)).cpu().numpy()
    rel = case.rel_blocks(got, ref)
    assert max(rel) <= 1e-11, rel


def test_jvp_fp32_parity(case):
    kk = lh_synth.normal_vector(case.gm.n, 4, 0.1)
    dk = lh_synth.normal_vector(case.gm.n, 5)
    tau = 0.02
    ref = case.hyd.jvp_complex_step(case.u, kk, tau, dk.astype(np.float32).astype(np.float64))
    got = case.gm.jvp(case.dev(case.u), case.dev(kk), tau, case.dev(dk, torch.float32)).double().cpu().numpy()
    rel = case.rel_blocks(got, ref)
    assert max(rel) <= 2e-5, rel


def test_jtvp_dot_product(case):
    """<J dk, y> = <dk, J^T y> for the GPU tangent and adjoint kernels."""
    kk = lh_synth.normal_vector(case.gm.n, 6, 0.1)
    dk = lh_synth.normal_vector(case.gm.n, 7)
    y = lh_synth.normal_vector(case.gm.n, 8)
    tau = 0.03
    u = case.dev(case.u)
    Jdk = case.gm.jvp(u, case.dev(kk), tau, case.dev(dk)).cpu().numpy()
    JTy = case.gm.jtvp(u, case.dev(kk), tau, case.dev(y)).cpu().numpy()
    a, b = float(Jdk @ y), float(dk @ JTy)
    scale = np.linalg.norm(Jdk) * np.linalg.norm(y)
    assert abs(a - b) <= 1e-13 * scale, (a, b)


@pytest.mark.parametrize("dim,n,k", [(2, (7, 5), 2), (3, (3, 3, 2), 2), (3, (2, 2, 1), 3)])
def test_negative_energy_parity(dim, n, k):
    """Eq. (19) on both branches: e ~ U(-1, 1), so about half of the quadrature points take
    the e < 0 evaluation of e+.  Residual, FP64 J.w, FP64 J^T.y and the record J.w against
    the oracle at the tolerances of the e >= 0 cases."""
    c = Case(dim, n, k, seed=31, visc=True, e_lo=-1.0)
    assert (c.u[2 * c.nx:] < 0).mean() > 0.3
    kk = lh_synth.normal_vector(c.gm.n, 32, 0.1)
    dk = lh_synth.normal_vector(c.gm.n, 33)
    tau = 0.01
    u, kd = c.dev(c.u), c.dev(kk)
    ref = c.hyd.residual(c.u, kk, tau)
    got = c.gm.residual(u, kd, tau).cpu().numpy()
    assert max(c.rel_blocks(got, ref)) <= 1e-12
    jref = c.hyd.jvp_complex_step(c.u, kk, tau, dk)
    got = c.gm.jvp(u, kd, tau, c.dev(dk)).cpu().numpy()
    assert max(c.rel_blocks(got, jref)) <= 1e-11
    jref32 = c.hyd.jvp_complex_step(c.u, kk, tau, dk.astype(np.float32).astype(np.float64))
    c.gm.linearize(u, kd, tau)
    got = c.gm.jvp(u, kd, tau, c.dev(dk, torch.float32), lin=True).double().cpu().numpy()
    assert max(c.rel_blocks(got, jref32)) <= 2e-5
    y = lh_synth.normal_vector(c.gm.n, 34)
    JTy = c.gm.jtvp(u, kd, tau, c.dev(y)).cpu().numpy()
    Jdk = c.gm.jvp(u, kd, tau, c.dev(dk)).cpu().numpy()
    assert abs(float(Jdk @ y) - float(dk @ JTy)) <= 1e-13 * np.linalg.norm(Jdk) * np.linalg.norm(y)


@pytest.mark.parametrize("dim,n,k,tg", [(2, (2, 2), 2, False), (2, (2, 1), 2, True), (3, (1, 1, 1), 2, False)])
def test_jtvp_dense_jacobian(dim, n, k, tg):
    """J^T y from the GPU adjoint against the oracle's dense complex-step Jacobian."""
    c = Case(dim, n, k, seed=21, visc=not tg, tg=tg)
    kk = lh_synth.normal_vector(c.gm.n, 9, 0.1)
    y = lh_synth.normal_vector(c.gm.n, 10)
    tau = 0.05
    Jd = c.hyd.jacobian(c.u, kk, tau)
    got = c.gm.jtvp(c.dev(c.u), c.dev(kk), tau, c.dev(y)).cpu().numpy()
    rel = c.rel_blocks(got, Jd.T @ y)
    assert max(rel) <= 1e-12, rel
    # and every column of J against the GPU tangent
    u, kd = c.dev(c.u), c.dev(kk)
    for j in range(0, c.gm.n, max(1, c.gm.n // 25)):
        e = np.zeros(c.gm.n)
        e[j] = 1.0
        col = c.gm.jvp(u, kd, tau, c.dev(e)).cpu().numpy()
        assert np.linalg.norm(col - Jd[:, j]) <= 1e-12 * max(1.0, np.linalg.norm(Jd[:, j]))


def test_mass_operators(case):
    m = case.hyd.m
    f = lh_synth.normal_vector(case.nx, 12).reshape(m.d, m.NV)
    ref = case.hyd.apply_mass_v(f).ravel()
    got = case.gm.mass_apply(0, case.dev(f.ravel())).cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    g = lh_synth.normal_vector(m.NEd, 13).reshape(m.NE, m.NL)
    ref = case.hyd.apply_mass_e(g).ravel()
    got = case.gm.mass_apply(1, case.dev(g.ravel())).cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    # solves: M_V by Jacobi-CG, M_E by its exact (diagonal) inverse
    Mv = case.hyd.mass_v_dense()
    rhs = lh_synth.normal_vector(case.nx, 14)
    sol, its = case.gm.mass_solve(0, case.dev(rhs), rtol=1e-13, maxit=1000)
    ref = np.linalg.solve(Mv, rhs.reshape(m.d, m.NV).T).T.ravel()
    assert its > 0 and np.linalg.norm(sol.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
    rhs_e = lh_synth.normal_vector(m.NEd, 15)
    sol_e, _ = case.gm.mass_solve(1, case.dev(rhs_e))
    ref_e = np.linalg.solve(case.hyd.mass_e_elem(), rhs_e.reshape(m.NE, m.NL, 1)).ravel()
    assert np.linalg.norm(sol_e.cpu().numpy() - ref_e) <= 1e-12 * np.linalg.norm(ref_e)


def test_energies(case):
    ke, ie = case.gm.energies(case.dev(case.u))
    assert abs(ke - case.hyd.kinetic_energy(case.u)) <= 1e-13 * abs(ke)
    assert abs(ie - case.hyd.internal_energy(case.u)) <= 1e-13 * abs(ie)


def test_jvp_fp32_record_parity(case):
    """FP32 J.w from the linearisation record (the point map linearised by the FP64 residual)."""
    import paper_2609_16424_b300 as lh
    kk = lh_synth.normal_vector(case.gm.n, 4, 0.1)
    dk = lh_synth.normal_vector(case.gm.n, 5)
    tau = 0.02
    ref = case.hyd.jvp_complex_step(case.u, kk, tau, dk.astype(np.float32).astype(np.float64))
    u, kd = case.dev(case.u), case.dev(kk)
    with pytest.raises(lh.LHError):
        case.gm.jvp(u, kd, tau, case.dev(dk, torch.float32), lin=True)
    case.gm.linearize(u, kd, tau)
    got = case.gm.jvp(u, kd, tau, case.dev(dk, torch.float32), lin=True).double().cpu().numpy()
    rel = case.rel_blocks(got, ref)
    assert max(rel) <= 2e-5, rel
    with pytest.raises(lh.LHError):          # a different tau is refused
        case.gm.jvp(u, kd, tau * 2, case.dev(dk, torch.float32), lin=True)


@pytest.mark.parametrize("dim,n,k", [(2, (6, 5), 2), (3, (4, 3, 3), 2), (2, (3, 4), 3)])
def test_kronecker_preconditioner_is_the_exact_block_inverse(dim, n, k):
    """P^-1 r: v rows = M_V^-1 restricted to free rows (uniform rho0), identity on fixed rows;
    x rows = r_x + tau z_v; e rows = M_E^-1 r_e."""
    c = Case(dim, n, k, seed=51)
    m = c.hyd.m
    r = lh_synth.normal_vector(c.gm.n, 52)
    tau = 0.037
    z = c.gm.precond(c.dev(r), tau).cpu().numpy()
    rx, rv, re = c.blocks(r)
    Mv = c.hyd.mass_v_dense()
    fixed = c.hyd.fixed
    zv = rv.reshape(m.d, m.NV).copy()
    for comp in range(m.d):
        f = ~fixed[comp]
        zv[comp, f] = np.linalg.solve(Mv[np.ix_(f, f)], rv.reshape(m.d, m.NV)[comp, f])
    zv = zv.ravel()
    ze = np.linalg.solve(c.hyd.mass_e_elem(), re.reshape(m.NE, m.NL, 1)).ravel()
    ref = np.concatenate([rx + tau * zv, zv, ze])
    rel = c.rel_blocks(z, ref)
    assert max(rel) <= 2e-6, rel


def test_jtvp_fp32_record(case):
    """FP32 transpose action from the record: against the FP64 adjoint (per block), and the
    dot-product identity with the FP32 record J.w."""
    kk = lh_synth.normal_vector(case.gm.n, 14, 0.1)
    y = lh_synth.normal_vector(case.gm.n, 15)
    dk = lh_synth.normal_vector(case.gm.n, 16)
    tau = 0.02
    u, kd = case.dev(case.u), case.dev(kk)
    ref = case.gm.jtvp(u, kd, tau, case.dev(y)).cpu().numpy()
    case.gm.linearize(u, kd, tau)
    yf = case.dev(y, torch.float32)
    got = case.gm.jtvp(u, kd, tau, yf, lin=True).double().cpu().numpy()
    rel = case.rel_blocks(got, ref)
    assert max(rel) <= 2e-5, rel
    dkf = case.dev(dk, torch.float32)
    jv = case.gm.jvp(u, kd, tau, dkf, lin=True).double()
    lhs = float((jv * yf.double()).sum())
    rhs = float((dkf.double() * case.gm.jtvp(u, kd, tau, yf, lin=True).double()).sum())
    scale = float((jv.abs() * yf.double().abs()).sum())
    assert abs(lhs - rhs) <= 1e-6 * scale
