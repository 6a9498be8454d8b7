"""Plain FP64 numpy MLP: the oracle of the surrogate network's kernels.

TEST INFRASTRUCTURE ONLY (imported by tests, never by the product).  The network is the
textbook fully connected net: a_{l+1} = GELU(a_l W_l^T + b_l) for hidden layers, the last
layer linear, GELU(x) = x Phi(x) with the exact normal CDF, loss = mean squared error over
all outputs; gradients by the chain rule written out layer by layer.  Parameter layout:
per layer W_l [out][in] row-major, then b_l (the same flat order the library uses).
"""
from __future__ import annotations

import math

import numpy as np

_SQRT2 = math.sqrt(2.0)


def _erf(x):
    return np.vectorize(math.erf)(x)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / _SQRT2))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / _SQRT2)) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def unpack(params, widths):
    p = np.asarray(params, np.float64)
    out, off = [], 0
    for l in range(len(widths) - 1):
        fi, fo = widths[l], widths[l + 1]
        W = p[off:off + fi * fo].reshape(fo, fi)
        off += fi * fo
        b = p[off:off + fo]
        off += fo
        out.append((W, b))
    assert off == p.size
    return out


def forward(params, widths, x):
    a = np.asarray(x, np.float64)
    layers = unpack(params, widths)
    zs, acts = [], [a]
    for l, (W, b) in enumerate(layers):
        z = acts[-1] @ W.T + b
        zs.append(z)
        acts.append(z if l == len(layers) - 1 else gelu(z))
    return acts[-1], zs, acts


def loss_and_grad(params, widths, x, t):
    y, zs, acts = forward(params, widths, x)
    t = np.asarray(t, np.float64)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    d = 2.0 * (y - t) / n
    grads = []
    layers = unpack(params, widths)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        if l != len(layers) - 1:
            d = d * gelu_grad(zs[l])
        grads.append((d.T @ acts[l], d.sum(axis=0)))
        d = d @ W
    flat = []
    for dW, db in reversed(grads):
        flat += [dW.ravel(), db]
    return loss, np.concatenate(flat)


def init_params(widths, seed: int) -> np.ndarray:
    """He-style uniform init from a seeded numpy generator (passed to the GPU as input)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(widths) - 1):
        fi, fo = widths[l], widths[l + 1]
        lim = math.sqrt(6.0 / fi)
        parts += [rng.uniform(-lim, lim, fo * fi), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)
