"""Learned Newton initial guess on the GPU: tensor-core MLP vs the FP64 oracle, feature and
completion layout, and the gain over plain extrapolation on held-out trajectories."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from oracle.fem import Mesh as OMesh

pytestmark = pytest.mark.gpu

DIMS = (341, 128, 3, 89)   # 3D Q2-Q1: inputs, hidden, hidden layers, outputs


def _net_and_data(seed, M=300):
    from paper_2609_16424_b300 import mlp
    rng = np.random.default_rng(seed)
    th = omlp.init_params(*DIMS, rng)
    net = mlp.MLP(DIMS[0], DIMS[1], DIMS[2], DIMS[3], params=th.astype(np.float32))
    X = rng.normal(size=(M, DIMS[0]))
    T = rng.normal(size=(M, DIMS[3])) * 0.3
    return net, th.astype(np.float32).astype(np.float64), X, T


def test_forward_matches_oracle():
    """BF16 operands, FP32 accumulation vs FP64: relative L2 <= 1e-2."""
    net, th, X, _ = _net_and_data(0)
    Y = net.forward(torch.tensor(X, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    ref, _ = omlp.forward(th, X, *DIMS)
    assert np.linalg.norm(Y - ref) <= 1e-2 * np.linalg.norm(ref)


def test_gradient_matches_oracle():
    """Loss within 1e-2 and every layer's gradient within 2e-2 (relative L2) of FP64."""
    net, th, X, T = _net_and_data(1)
    loss, g = net.grad(torch.tensor(X, dtype=torch.float32, device="cuda"),
                       torch.tensor(T, dtype=torch.float32, device="cuda"))
    lref, gref = omlp.loss_and_grad(th, X, T, *DIMS)
    assert abs(loss - lref) <= 1e-2 * lref
    g = g.double().cpu().numpy()
    o = 0
    for (r, c) in omlp.shapes(*DIMS):
        for size in (r * c, r):
            a, b = g[o:o + size], gref[o:o + size]
            assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b), (o, size)
            o += size


def test_adam_training_reduces_loss():
    net, _, X, _ = _net_and_data(2, M=4096)
    A = np.random.default_rng(3).normal(size=(DIMS[0], DIMS[3])) / np.sqrt(DIMS[0])
    T = np.tanh(X @ A)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    l0 = net.train_step(Xd, Td, 1e-3)
    for _ in range(150):
        last = net.train_step(Xd, Td, 1e-3)
    assert last < 0.3 * l0


def test_features_and_completion_layout():
    """Feature rows are the element dofs of k1, k2 (scaled) and dt; the initial guess has
    v rows = k1 + nodal mean of the element predictions (0 on walls), e rows = k1 + own
    prediction, x rows = u_v + tau k0_v."""
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300 import mlp
    dim, n, k = 3, (3, 2, 2), 2
    om = OMesh(n, (0,) * 3, (1,) * 3, k)
    gm = lh.Mesh(dim, n, (0,) * 3, (1,) * 3, k)
    rng = np.random.default_rng(4)
    k1, k2, u = (rng.normal(size=gm.n) for _ in range(3))
    scale = torch.tensor([2.0, 3.0, 5.0, 0.1], dtype=torch.float32, device="cuda")
    d = lambda a: torch.tensor(a, device="cuda")
    X = mlp.features(gm, d(k1), d(k2), 0.02, scale).double().cpu().numpy()
    nd, nl = om.ND, om.NL

    def elem_rows(kv):
        x, v, e = om.split(kv)
        return np.concatenate([om.gather(x).reshape(om.NE, -1) / 2.0, om.gather(v).reshape(om.NE, -1) / 3.0,
                               e / 5.0], axis=1)
    ref = np.concatenate([elem_rows(k1), elem_rows(k2), np.full((om.NE, 1), 0.2)], axis=1)
    assert np.allclose(X, ref, rtol=1e-6, atol=1e-6)
    Y = rng.normal(size=(om.NE, dim * nd + nl)).astype(np.float32)
    tau = 0.013
    k0 = mlp.apply(gm, d(u), tau, d(k1), torch.tensor(Y, device="cuda"), scale).cpu().numpy()
    yv = Y[:, :dim * nd].reshape(om.NE, dim, nd).transpose(1, 0, 2).astype(np.float64) * 3.0
    cnt = np.zeros(om.NV)
    np.add.at(cnt, om.conn, 1.0)
    dv = np.zeros((dim, om.NV))
    for c in range(dim):
        np.add.at(dv[c], om.conn, yv[c])
    _, k1v, k1e = om.split(k1)
    kv = np.where(om.boundary_mask(0x3f), 0.0, k1v + dv / cnt)
    ke = k1e + Y[:, dim * nd:].astype(np.float64) * 5.0
    _, uv, _ = om.split(u)
    ref0 = om.join(uv + tau * kv, kv, ke)
    assert np.allclose(k0, ref0, rtol=1e-6, atol=1e-6)


def _family(make, nrun, steps, ntrain, dim, k, cfl):
    """Seeded trajectories of a problem family, a network trained on the first ntrain runs,
    and the held-out runs (Newton rtol 1e-8 for the training data, FP32 J.w)."""
    from paper_2609_16424_b300 import mlp
    newton = dict(newton_rtol=1e-8, gmres_rtol=1e-4, gmres_maxit=200, restart=30, jvp_prec="fp32")
    runs = []
    for i in range(nrun):
        gm, u0 = make(i)
        runs.append((gm, u0, mlp.trajectory(gm, u0, steps, cfl=cfl, **newton)))
    gm0 = runs[0][0]
    train = [tr for _, _, tr in runs[:ntrain]]
    fscale = torch.zeros(4, dtype=torch.float32, device="cuda")
    fscale[:3] = mlp.group_rms(gm0, [kk for tr in train for _, kk in tr]).float()
    fscale[3] = float(np.mean([dt for tr in train for dt, _ in tr]))
    tscale = torch.ones(4, dtype=torch.float32, device="cuda")
    tscale[:3] = mlp.group_rms(gm0, [tr[i][1] - tr[i - 1][1] for tr in train for i in range(1, len(tr))]).float()
    X, T = mlp.dataset(gm0, train, fscale, tscale)
    n_in, n_out = mlp.feature_sizes(dim, k)
    net = mlp.MLP(n_in, 128, 3, n_out, seed=1)
    mlp.train(net, X, T, epochs=40)
    return net, fscale, tscale, runs[ntrain:]


def _evaluate(net, fscale, tscale, heldout, tol):
    """On held-out steps: initial-residual and error ratios of the proposal against plain
    extrapolation, and Newton / GMRES iterations of both guesses to one absolute tolerance,
    tol x ||R(k^{n-1})|| (the paper's relative tolerance 1e-5, measured against the fallback's
    initial residual, so that both guesses stop at the same accuracy)."""
    from paper_2609_16424_b300 import mlp
    ratios_r, ratios_e, its, gits = [], [], [], []
    for gm, u0, tr in heldout:
        u = u0.clone()
        for i, (dt, kn) in enumerate(tr):
            tau = 0.5 * dt
            if i >= 2:
                k1, k2 = tr[i - 1][1], tr[i - 2][1]
                k0 = mlp.apply(gm, u, tau, k1, net.forward(mlp.features(gm, k1, k2, dt, fscale)), tscale)
                r1 = float(gm.residual(u, k1, tau).norm())
                ratios_r.append(float(gm.residual(u, k0, tau).norm()) / r1)
                ratios_e.append(float((k0 - kn).norm() / (k1 - kn).norm()))
                pair, gpair = [], []
                for guess in (k1, k0):
                    st = gm.newton_step(u.clone(), guess.clone(), dt, newton_rtol=1e-30, newton_atol=tol * r1,
                                        gmres_rtol=1e-4, gmres_maxit=200, restart=30, jvp_prec="fp32")
                    pair.append(st["newton_its"])
                    gpair.append(st["gmres_its_total"])
                its.append(pair)
                gits.append(gpair)
            u = u + dt * kn
    return np.mean(ratios_r), np.mean(ratios_e), np.mean(its, axis=0), np.mean(gits, axis=0)


def test_learned_proposal_on_heldout_blasts():
    """3D point blasts (the 24^3 benchmark family at 8^3), seeded gamma in [1.3, 1.7] and
    deposits in [0.1, 0.5], 6 training runs, 2 held out.  The proposal's initial residual and
    its distance to the converged increment are well below plain extrapolation's.  Measured
    (not asserted): at the paper's tolerance it saves no Newton iteration and GMRES needs more
    iterations than from extrapolation, so it does not pay on this family."""
    import paper_2609_16424_b300 as lh
    from paper_2609_16424_b300.states import blast_state
    rng = np.random.default_rng(0)
    params = [(rng.uniform(1.3, 1.7), rng.uniform(0.1, 0.5)) for _ in range(8)]

    def make(i):
        gm = lh.Mesh(3, (8, 8, 8), (0,) * 3, (1,) * 3, 2, gamma=params[i][0])
        return gm, blast_state(gm, params[i][1])
    net, fs, ts, held = _family(make, 8, 24, 6, 3, 2, 2.0)
    rr, re, its, gits = _evaluate(net, fs, ts, held, 1e-5)
    print("blast: residual ratio", rr, "error ratio", re, "newton", its, "gmres", gits)
    assert rr < 0.2 and re < 0.7


def test_learned_proposal_gains_on_taylor_green():
    """2D Taylor-Green vortex, 16 x 16 Q2-Q1, seeded velocity amplitudes in [0.5, 1.5] and
    pressure levels p0 in [1, 10], implicit midpoint at FS-CFL 8; 6 training runs, 2 held out.
    At the paper's tolerance the proposal takes fewer Newton iterations per step than plain
    extrapolation.  GMRES iterations are reported, not asserted: on this family they drop,
    but over 160 training and 39 held-out runs (bench.py --mlp) they grow, and the step is
    slower than with extrapolation."""
    from paper_2609_16424_b300.states import taylor_green_problem
    rng = np.random.default_rng(1)
    params = [(rng.uniform(0.5, 1.5), rng.uniform(1.0, 10.0)) for _ in range(8)]

    def make(i):
        gm, u = taylor_green_problem(16, 2, p0=params[i][1], device="cuda:0")
        u[2 * gm.NV:4 * gm.NV] *= params[i][0]
        return gm, u
    net, fs, ts, held = _family(make, 8, 24, 6, 2, 2, 8.0)
    rr, re, its, gits = _evaluate(net, fs, ts, held, 1e-5)
    print("taylor-green: residual ratio", rr, "error ratio", re, "newton", its, "gmres", gits)
    assert rr < 0.2 and re < 0.7
    assert its[1] < its[0], (its, gits)
