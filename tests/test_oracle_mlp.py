"""Pins of the oracle MLP: central-difference gradients, GELU values, Adam's first step."""
import numpy as np

from oracle import mlp


def test_gelu_values():
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(8.0)) - 8.0) < 1e-12          # Phi(8) = 1 - 6e-16
    assert abs(mlp.gelu(np.array(-8.0))) < 1e-12
    assert abs(mlp.gelu_grad(np.array(0.0)) - 0.5) < 1e-15       # Phi(0) = 1/2
    z = np.linspace(-3, 3, 13)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_gradient_against_central_differences():
    rng = np.random.default_rng(0)
    dims = (7, 6, 2, 5)
    th = mlp.init_params(*dims, rng)
    X = rng.normal(size=(9, 7))
    T = rng.normal(size=(9, 5))
    _, g = mlp.loss_and_grad(th, X, T, *dims)
    h = 1e-6
    for i in rng.choice(th.size, 40, replace=False):
        e = np.zeros_like(th)
        e[i] = h
        fd = (mlp.loss_and_grad(th + e, X, T, *dims)[0] - mlp.loss_and_grad(th - e, X, T, *dims)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_first_adam_step_is_lr_times_sign():
    """With bias correction the first update is lr * g / (|g| + eps) = lr * sign(g)."""
    opt = mlp.Adam(4, lr=0.01)
    g = np.array([3.0, -0.2, 1e-3, -7.0])
    th = opt.step(np.zeros(4), g)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-4)


def test_training_reduces_loss():
    rng = np.random.default_rng(1)
    dims = (3, 16, 2, 2)
    th = mlp.init_params(*dims, rng)
    X = rng.normal(size=(64, 3))
    T = np.stack([np.sin(X[:, 0]) + X[:, 1], X[:, 2] ** 2], axis=1)
    opt = mlp.Adam(th.size, lr=1e-2)
    l0 = mlp.loss_and_grad(th, X, T, *dims)[0]
    for _ in range(300):
        _, g = mlp.loss_and_grad(th, X, T, *dims)
        th = opt.step(th, g)
    assert mlp.loss_and_grad(th, X, T, *dims)[0] < 0.2 * l0
