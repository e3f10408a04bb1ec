"""The explicit comparison path on the GPU against the oracle (oracle/explicit.py): F's two
applications (F.1 and F^T w + b) with the smooth viscosity mu_imp and the original tensor
viscosity mu_exp, the explicit time-step estimate, single RK2-average / RK3 / RK4 steps,
a run with the explicit step control, and exact energy conservation of RK2-average.

Tolerances: F.1 and F^T w relative L2 <= 1e-12 (mu_imp) / 1e-11 (mu_exp: the eigenpair is
computed in closed form on the GPU and by LAPACK in the oracle); steps <= 1e-11 per block
(the M_V solves stop at 1e-13); the estimate <= 1e-12."""
import numpy as np
import pytest
import torch

import lh_synth
from lhcase import Case
from oracle.explicit import Explicit, dt_estimate, explicit_advance, explicit_step, total_energy

pytestmark = pytest.mark.gpu

CASES = [
    (2, (5, 4), 1, True, False),
    (2, (4, 3), 2, True, False),
    (2, (4, 3), 2, False, True),     # Taylor-Green source, no viscosity
    (2, (3, 2), 3, True, False),
    (2, (2, 2), 4, True, False),
    (2, (3, 3), 3, False, True),     # Taylor-Green source at Q3-Q2
    (3, (3, 2, 2), 1, True, False),
    (3, (2, 2, 2), 2, True, False),
    (3, (2, 1, 1), 3, True, False),
]
IDS = [f"d{c[0]}_n{'x'.join(map(str, c[1]))}_k{c[2]}{'_visc' if c[3] else ''}{'_tg' if c[4] else ''}" for c in CASES]
TOL = {"imp": 1e-12, "exp": 1e-11}


def _case(param, model, seed=41):
    dim, n, k, visc, tg = param
    return Case(dim, n, k, seed=seed, visc=visc, tg=tg, gamma=5.0 / 3.0 if tg else 1.4, visc_model=model)


@pytest.mark.parametrize("model", ["imp", "exp"])
@pytest.mark.parametrize("param", CASES, ids=IDS)
def test_force_and_estimate_parity(param, model):
    c = _case(param, model)
    ex = Explicit(c.hyd)
    m = c.hyd.m
    Fb = ex.assemble(c.u)
    w = lh_synth.normal_vector(m.d * m.NV, 7).reshape(m.d, m.NV)
    ref1 = ex.f_one(Fb).ravel()
    reft = ex.f_t(Fb, w).ravel()
    f1, ftw, est = c.gm.force(c.dev(c.u), c.dev(w.ravel()), estimate=True, visc_model=model)
    f1, ftw = f1.cpu().numpy(), ftw.cpu().numpy()
    assert np.linalg.norm(f1 - ref1) <= TOL[model] * np.linalg.norm(ref1)
    assert np.linalg.norm(ftw - reft) <= TOL[model] * np.linalg.norm(reft)
    ref_est = dt_estimate(c.hyd, c.u)
    assert abs(est - ref_est) <= 1e-12 * ref_est


@pytest.mark.parametrize("scheme", [2, 3, 4])
@pytest.mark.parametrize("model", ["imp", "exp"])
@pytest.mark.parametrize("param", [CASES[1], CASES[2], CASES[5], CASES[7]], ids=[IDS[1], IDS[2], IDS[5], IDS[7]])
def test_explicit_step_parity(param, model, scheme):
    c = _case(param, model)
    dt = 0.2 * dt_estimate(c.hyd, c.u)
    ref = explicit_step(Explicit(c.hyd), c.u, dt, scheme)
    u = c.dev(c.u)
    st = c.gm.explicit_step(u, dt, scheme=scheme, visc_model=model)
    rel = c.rel_blocks(u.cpu().numpy(), ref)
    assert max(rel) <= 1e-11, rel
    assert st["force_evals"] == (2 if scheme == 2 else scheme)


def _blast(dim, n, k, model):
    c = Case(dim, (n,) * dim, k, seed=1, visc=True, visc_model=model)
    m = c.hyd.m
    e = np.zeros((m.NE, m.NL)) + 0.01
    e[0, :] = 0.5 * m.NE
    u = m.join(c.hyd.x0, np.zeros((dim, m.NV)), e)
    return c, u


@pytest.mark.parametrize("model", ["imp", "exp"])
def test_explicit_run_with_step_control_matches_oracle(model):
    """Same accepted and repeated steps as the oracle's run, same final state."""
    c, u0 = _blast(2, 4, 2, model)
    ref, steps, rejected = explicit_advance(c.hyd, u0, 0.05, 0.3, 2)
    u = c.dev(u0)
    st = c.gm.explicit_advance(u, 0.05, cfl=0.3, scheme=2, visc_model=model)
    assert (st["steps"], st["rejected"]) == (steps, rejected)
    rel = c.rel_blocks(u.cpu().numpy(), ref)
    assert max(rel) <= 1e-9, rel


def test_rk2_average_conserves_energy_on_the_gpu():
    c, u0 = _blast(3, 5, 2, "exp")
    u = c.dev(u0)
    ke0, ie0 = c.gm.energies(u)
    st = c.gm.explicit_advance(u, 0.05, cfl=0.5, scheme=2, visc_model="exp")
    ke, ie = c.gm.energies(u)
    assert st["steps"] >= 3 and ke > 1e-3 * ie
    assert abs(ke + ie - ke0 - ie0) <= 1e-12 * (ke0 + ie0)
    assert abs(total_energy(c.hyd, u.cpu().numpy()) - (ke0 + ie0)) <= 1e-12 * (ke0 + ie0)
