"""Pins of the FP64 oracle MLP (CPU): GELU against scipy's erf and its limits, the
chain-rule gradients against central finite differences of the loss."""
import numpy as np
import scipy.special as sp

from oracle import mlp


def test_gelu_definition_and_limits():
    x = np.linspace(-6, 6, 61)
    assert np.allclose(mlp.gelu(x), 0.5 * x * (1 + sp.erf(x / np.sqrt(2))), atol=1e-15)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([40.0]))[0] - 40.0) < 1e-12
    assert abs(mlp.gelu(np.array([-40.0]))[0]) < 1e-12
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_gradients_equal_finite_differences():
    widths = [3, 5, 4, 2]
    rng = np.random.default_rng(0)
    p = mlp.init_params(widths, 1).astype(np.float64) + 0.05 * rng.standard_normal(
        sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(3)))
    x = rng.standard_normal((7, 3))
    t = rng.standard_normal((7, 2))
    loss, g = mlp.loss_and_grad(p, widths, x, t)
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss_and_grad(p + e, widths, x, t)[0] - mlp.loss_and_grad(p - e, widths, x, t)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    y, _, _ = mlp.forward(p, widths, x)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-15
