"""Learned Newton initial guess (argument marshalling over the lh_mlp_* C calls).

Workflow of one implicit step with the proposal:
    X  = features(mesh, k1, k2, dt)        # k1 = k^{n-1}, k2 = k^{n-2}   (lh_mlp_features)
    Y  = net.forward(X)                    # per-element correction        (lh_mlp_forward)
    k0 = apply(mesh, k1, Y)                # nodal average, k0 = k1 + dk   (lh_mlp_apply_prediction)
    mesh.newton_step(u, k0, dt)            # k0 is the initial guess; k0 <- converged k
Plain extrapolation is k0 = k1; both are measured against the converged k.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib
from . import lib as _L
from .hydro import LHError


def _p(t):
    return C.c_void_p(t.data_ptr())


class MLP:
    """Per-element network on the GPU (BF16 tensor-core matmuls, FP32 accumulation/master)."""

    def __init__(self, n_in, hidden=128, layers=3, n_out=None, params=None, seed=0, device="cuda"):
        self.n_in, self.hidden, self.layers, self.n_out = n_in, hidden, layers, n_out
        self.device = torch.device(device)
        if params is None:
            params = init_params(n_in, hidden, layers, n_out, np.random.default_rng(seed))
        host = np.ascontiguousarray(params, dtype=np.float32)
        h = C.c_void_p()
        st = _L.lh_mlp_create(n_in, hidden, layers, n_out, host.ctypes.data_as(C.c_void_p),
                              C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream), C.byref(h))
        if st != _lib.LH_OK:
            raise LHError(st, _L.lh_last_error(None).decode())
        self._h = h
        self.n_params = int(_L.lh_mlp_num_params(h))
        assert self.n_params == host.size

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _L.lh_mlp_destroy(h)
            self._h = None

    def _check(self, st):
        if st != _lib.LH_OK:
            raise LHError(st, _L.lh_mlp_last_error(self._h).decode())

    def params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        self._check(_L.lh_mlp_params(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def forward(self, X):
        X = X.contiguous()
        Y = torch.empty(X.shape[0], self.n_out, dtype=torch.float32, device=self.device)
        self._check(_L.lh_mlp_forward(self._h, _p(X), X.shape[0], _p(Y)))
        return Y

    def grad(self, X, T):
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        loss = C.c_double()
        self._check(_L.lh_mlp_grad(self._h, _p(X.contiguous()), _p(T.contiguous()), X.shape[0], _p(g),
                                   C.byref(loss)))
        return loss.value, g

    def train_step(self, X, T, lr):
        loss = C.c_double()
        self._check(_L.lh_mlp_train_step(self._h, _p(X.contiguous()), _p(T.contiguous()), X.shape[0],
                                         C.c_float(lr), C.byref(loss)))
        return loss.value


def init_params(n_in, hidden, layers, n_out, rng):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, in the flat layout."""
    dims = [n_in] + [hidden] * layers + [n_out]
    parts = []
    for i in range(len(dims) - 1):
        a = 1.0 / np.sqrt(dims[i])
        parts += [rng.uniform(-a, a, size=dims[i + 1] * dims[i]), rng.uniform(-a, a, size=dims[i + 1])]
    return np.concatenate(parts).astype(np.float32)


def feature_sizes(dim, k):
    """(network inputs, network outputs): inputs = element dofs [x | v | e] of the last two
    increments and dt; outputs = corrections of the v and e rows (x rows follow exactly)."""
    nd, nl = (k + 1) ** dim, k ** dim
    f1 = 2 * dim * nd + nl
    return 2 * f1 + 1, dim * nd + nl


def features(mesh, k1, k2, dt, scale):
    n_in, _ = feature_sizes(mesh.dim, mesh.order)
    X = torch.empty(mesh.NE, n_in, dtype=torch.float32, device=mesh.device)
    mesh._stream()
    st = _L.lh_mlp_features(mesh._h, _p(k1), _p(k2), C.c_double(dt), _p(scale), _p(X))
    if st != _lib.LH_OK:
        raise LHError(st, _L.lh_last_error(None).decode())
    return X


def apply(mesh, u, tau, k1, Y, scale):
    """Initial guess k0 at (u, tau): v and e rows from the prediction, x rows exact."""
    k0 = torch.empty_like(k1)
    mesh._stream()
    st = _L.lh_mlp_apply_prediction(mesh._h, _p(u), C.c_double(tau), _p(k1), _p(Y.contiguous()), _p(scale),
                                    _p(k0))
    if st != _lib.LH_OK:
        raise LHError(st, _L.lh_last_error(None).decode())
    return k0


def element_targets(mesh, k_new, k1, scale):
    """Training targets per element: element dofs of the v and e rows of (k_new - k1),
    scaled by scale[1] / scale[2] (the correction the network predicts)."""
    nd = (mesh.order + 1) ** mesh.dim
    zero = torch.zeros_like(k1)
    X = features(mesh, k_new - k1, zero, 0.0, scale)
    f1 = 2 * mesh.dim * nd + mesh.order ** mesh.dim
    return X[:, mesh.dim * nd:f1].contiguous()


def trajectory(mesh, u0, steps, cfl=2.0, **newton_kw):
    """Implicit midpoint steps from u0 with dt = cfl * explicit estimate; returns the
    converged increments and time steps [(dt_n, k_n)] (the proposal's training data)."""
    u = u0.clone()
    k = torch.zeros_like(u)
    out = []
    for _ in range(steps):
        dt = cfl * mesh.dt_estimate(u)
        mesh.newton_step(u, k, dt, **newton_kw)
        out.append((dt, k.clone()))
    return out


def group_rms(mesh, vecs):
    """RMS of the x, v and e rows over a list of increments (feature / target scales)."""
    nx = mesh.dim * mesh.NV
    acc = torch.zeros(3, dtype=torch.float64, device=mesh.device)
    cnt = torch.zeros(3, dtype=torch.float64, device=mesh.device)
    for v in vecs:
        for g, sl in enumerate((slice(0, nx), slice(nx, 2 * nx), slice(2 * nx, mesh.n))):
            acc[g] += (v[sl] ** 2).sum()
            cnt[g] += v[sl].numel()
    r = torch.sqrt(acc / cnt)
    return torch.where(r > 0, r, torch.ones_like(r))


def dataset(mesh, trajs, fscale, tscale):
    """Element samples (X, T) from trajectories: inputs k^{n-1}, k^{n-2}, dt_n; target the
    scaled correction k^n - k^{n-1}."""
    Xs, Ts = [], []
    for traj in trajs:
        for n in range(2, len(traj)):
            dt, kn = traj[n]
            Xs.append(features(mesh, traj[n - 1][1], traj[n - 2][1], dt, fscale))
            Ts.append(element_targets(mesh, kn, traj[n - 1][1], tscale))
    return torch.cat(Xs), torch.cat(Ts)


def train(net, X, T, epochs=40, batch=2048, lr=1e-3, seed=0):
    """Mini-batch Adam over shuffled element samples; returns the loss history per epoch."""
    g = torch.Generator(device=X.device).manual_seed(seed)
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(X.shape[0], generator=g, device=X.device)
        tot, nb = 0.0, 0
        for i in range(0, X.shape[0] - batch + 1, batch):
            idx = perm[i:i + batch]
            tot += net.train_step(X[idx], T[idx], lr)
            nb += 1
        hist.append(tot / max(nb, 1))
    return hist
