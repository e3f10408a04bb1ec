"""FP64 reference of the per-element MLP that proposes the Newton initial guess.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The learned proposal is an addition
to the paper's method: the paper initialises each stage solve from the previous stage
increment (Sec. 3.5 leaves the initial guess open); the network predicts the correction
k^n - k^{n-1} per element from the element dofs of the last two increments and dt.

Network: Linear(in, h) -> GELU -> [Linear(h, h) -> GELU] x (L - 1) -> Linear(h, out), with
GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 (exact form), mean-squared-error loss over
all outputs, Adam (Kingma & Ba 2015) with bias correction.  Parameters are flat in the
order W_1 [h][in], b_1 [h], ..., W_L+1 [out][h], b_L+1 [out] (the GPU layout).

Pinned by tests/test_oracle_mlp.py: gradients against central differences, GELU limits
and derivative at 0, the first Adam step equals lr * sign(g), loss decrease on a fit.
"""
import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def shapes(n_in, hidden, layers, n_out):
    dims = [n_in] + [hidden] * layers + [n_out]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def unpack(theta, n_in, hidden, layers, n_out):
    out, o = [], 0
    for (r, c) in shapes(n_in, hidden, layers, n_out):
        W = theta[o:o + r * c].reshape(r, c)
        o += r * c
        b = theta[o:o + r]
        o += r
        out.append((W, b))
    assert o == theta.size
    return out


def n_params(n_in, hidden, layers, n_out):
    return sum(r * c + r for (r, c) in shapes(n_in, hidden, layers, n_out))


def forward(theta, X, n_in, hidden, layers, n_out):
    """Returns Y and the cache (inputs and pre-activations of every layer)."""
    Ws = unpack(theta, n_in, hidden, layers, n_out)
    H, cache = X, []
    for i, (W, b) in enumerate(Ws):
        Z = H @ W.T + b
        cache.append((H, Z))
        H = gelu(Z) if i < len(Ws) - 1 else Z
    return H, cache


def loss_and_grad(theta, X, T, n_in, hidden, layers, n_out):
    """Mean squared error over all outputs and its gradient w.r.t. theta."""
    Ws = unpack(theta, n_in, hidden, layers, n_out)
    Y, cache = forward(theta, X, n_in, hidden, layers, n_out)
    R = Y - T
    loss = float(np.mean(R * R))
    dZ = 2.0 * R / R.size
    grads = []
    for i in range(len(Ws) - 1, -1, -1):
        H, Z = cache[i]
        W, _ = Ws[i]
        if i < len(Ws) - 1:
            dZ = dZ * gelu_grad(Z)
        grads.append((dZ.T @ H, dZ.sum(axis=0)))
        dZ = dZ @ W
    g = []
    for dW, db in reversed(grads):
        g += [dW.ravel(), db]
    return loss, np.concatenate(g)


class Adam:
    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m, self.v, self.t = np.zeros(n), np.zeros(n), 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def init_params(n_in, hidden, layers, n_out, rng):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    parts = []
    for (r, c) in shapes(n_in, hidden, layers, n_out):
        a = 1.0 / np.sqrt(c)
        parts += [rng.uniform(-a, a, size=r * c), rng.uniform(-a, a, size=r)]
    return np.concatenate(parts)
