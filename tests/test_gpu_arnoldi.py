"""Device-driven Arnoldi of the FP32-basis GMRES (each restart cycle one CUDA graph launch
whose WHILE node repeats the Arnoldi iteration, with the Givens rotations and the stopping
test on the device) against the host loop (one read-back per iteration): the same
Newton-GMRES iterations and the same step, for every preconditioner kind, with restarts,
with the row-scaled norm and with the tensor-core J.w; and the driver's fallback rules."""
import numpy as np
import pytest
import torch

from lhcase import Case

pytestmark = pytest.mark.gpu


def _steps(c, u0, arnoldi, nsteps=3, dt=0.01, **kw):
    """nsteps implicit midpoint steps from u0 (the first GMRES solve of a new operator kind
    runs on the host; the later ones take the device path when arnoldi = 1)."""
    u, k = u0.clone(), torch.zeros_like(u0)
    its = []
    for _ in range(nsteps):
        st = c.gm.newton_step(u, k, dt, arnoldi=arnoldi, **kw)
        its.append((st["newton_its"], st["gmres_its_total"], st["jvp_evals"]))
    return u.cpu().numpy(), its


@pytest.mark.parametrize("opts", [
    dict(precond="kron"),
    dict(precond="jacobi"),
    dict(precond="jvv_diag"),
    dict(precond="cheb", cheb_degree=3),
    dict(precond="kron", restart=4),                     # several restart cycles per solve
    dict(precond="kron", scaled_norm=1),
    dict(precond="kron", jvp_prec="bf16"),
])
def test_device_arnoldi_matches_host_loop(opts):
    c = Case(3, (4, 4, 4), 2, seed=11, vscale=1.0)
    u0 = c.dev(c.u)
    kw = dict(newton_rtol=1e-10, gmres_rtol=1e-6, gmres_maxit=300, restart=30, jvp_prec="fp32")
    kw.update(opts)
    a, ia = _steps(c, u0, 0, **kw)
    b, ib = _steps(c, u0, 1, **kw)
    # the same arithmetic up to the rounding of the Givens rotations (device vs host hypot)
    assert ia == ib, (ia, ib)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a), np.linalg.norm(a - b)


def test_device_arnoldi_2d_and_iteration_budget():
    """2D Q3 (another element kernel in the recorded body) and a GMRES budget that ends a
    cycle early (stop by the iteration budget, not by convergence)."""
    c = Case(2, (6, 6), 3, seed=4, vscale=1.0)
    u0 = c.dev(c.u)
    kw = dict(newton_rtol=1e-6, gmres_rtol=1e-8, gmres_maxit=7, restart=5, jvp_prec="fp32", newton_maxit=30)
    a, ia = _steps(c, u0, 0, nsteps=2, **kw)
    b, ib = _steps(c, u0, 1, nsteps=2, **kw)
    assert ia == ib, (ia, ib)
    assert all(g <= 7 * n for n, g, _ in ia)   # every solve stopped within its 7 iterations
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)


def test_device_arnoldi_rejects_bad_option():
    import paper_2609_16424_b300 as lh
    c = Case(2, (2, 2), 2, seed=1)
    u = c.dev(c.u)
    with pytest.raises(lh.LHError) as ei:
        c.gm.newton_step(u.clone(), torch.zeros_like(u), 0.01, jvp_prec="fp32", arnoldi=2)
    assert ei.value.status == 1


def test_device_arnoldi_rerecords_on_new_step_size_and_per_mesh():
    """The recorded cycle depends on tau (= dt / 2): steps of changing dt re-record it, and two
    meshes used alternately each keep their own; both must still match the host loop."""
    ca = Case(3, (4, 4, 4), 2, seed=11, vscale=1.0)
    cb = Case(2, (8, 6), 2, seed=12, vscale=1.0)
    kw = dict(newton_rtol=1e-10, gmres_rtol=1e-6, gmres_maxit=300, restart=30, jvp_prec="fp32")
    dts = (0.01, 0.007, 0.013, 0.007)

    def run(arnoldi):
        ua, ka = ca.dev(ca.u), torch.zeros(ca.u.size, dtype=torch.float64, device="cuda")
        ub, kb = cb.dev(cb.u), torch.zeros(cb.u.size, dtype=torch.float64, device="cuda")
        its = []
        for dt in dts:
            sa = ca.gm.newton_step(ua, ka, dt, arnoldi=arnoldi, **kw)
            sb = cb.gm.newton_step(ub, kb, 0.5 * dt, arnoldi=arnoldi, **kw)
            its.append((sa["gmres_its_total"], sb["gmres_its_total"]))
        return ua.cpu().numpy(), ub.cpu().numpy(), its

    a0, b0, i0 = run(0)
    a1, b1, i1 = run(1)
    assert i0 == i1, (i0, i1)
    assert np.linalg.norm(a1 - a0) <= 1e-10 * np.linalg.norm(a0)
    assert np.linalg.norm(b1 - b0) <= 1e-10 * np.linalg.norm(b0)
