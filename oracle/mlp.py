"""Oracle of the threshold-picker MLP -- TEST INFRASTRUCTURE ONLY.

Float64 numpy statement of the network the CUDA picker trains: 66 inputs ->
128 (ReLU) -> 128 (ReLU) -> 1 output, loss = mean squared error, Adam
(Kingma & Ba 2015) with bias correction.  The paper has no learned picker
(it chooses thresholds by rules of thumb, Sec. IV-D); the architecture is the
project's.  A second objective, the soft-level ARI loss, mixes the squared
error with the expected ARI lost by a Gaussian-smoothed level choice.
Parameter vector layout: W1 [128 x 66] row-major, b1 [128], W2 [128 x 128],
b2 [128], w3 [128], b3 [1].

Parity unpinned by the paper: pinned by finite differences, closed forms and
the Adam first-step identity (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

IN, HID = 66, 128
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("w3", (HID,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, at = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[at:at + size].reshape(shape)
        at += size
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(theta, X):
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, target):
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(target, dtype=np.float64)) ** 2))


def _backprop(p, dy, X, z1, h1, z2, h2):
    """Gradient of every parameter from dloss/dy by the chain rule."""
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return pack(g)


def loss_and_grad(theta, X, target):
    """Loss and its gradient by the chain rule (backpropagation)."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    dy = 2.0 * (y - np.asarray(target, dtype=np.float64)) / n
    return float(np.mean((y - target) ** 2)), _backprop(p, dy, X, z1, h1, z2, h2)


def soft_level_loss(y, L, sigma):
    """Expected ARI loss of a smoothed level choice, per sample, and its
    derivative in y.  The picker's level is round(64 y); here every grid
    level i = 1..64 gets the weight w_i ~ exp(-(i - 64 y)^2 / (2 sigma^2))
    (normalised to sum 1), and the loss is sum_i w_i L_i, L_i the ARI lost at
    level i against the best level (L: N x 64).  As sigma -> 0 it tends to the
    ARI lost at the nearest level.  d/dy = 64 / sigma^2 *
    (sum_i w_i L_i (i - p) - loss * sum_i w_i (i - p)), p = 64 y."""
    y = np.asarray(y, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    i = np.arange(1, L.shape[1] + 1, dtype=np.float64)
    d = i[None, :] - 64.0 * y[:, None]
    a = -d * d / (2.0 * sigma * sigma)
    w = np.exp(a - a.max(axis=1, keepdims=True))
    w /= w.sum(axis=1, keepdims=True)
    val = (w * L).sum(axis=1)
    dval = 64.0 / (sigma * sigma) * ((w * L * d).sum(axis=1) - val * (w * d).sum(axis=1))
    return val, dval


def mixed_loss_and_grad(theta, X, target, L, sigma, mix):
    """mix * (mean squared error to target) + (1 - mix) * (mean soft-level
    ARI loss), and its gradient by backpropagation."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    t = np.asarray(target, dtype=np.float64)
    sv, sd = soft_level_loss(y, L, sigma)
    dy = (mix * 2.0 * (y - t) + (1.0 - mix) * sd) / n
    return float(np.mean(mix * (y - t) ** 2 + (1.0 - mix) * sv)), _backprop(p, dy, X, z1, h1, z2, h2)


def adam(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1): returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init(seed: int):
    """Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = {}
    for name, shape in SHAPES:
        if name.startswith("b"):
            parts[name] = np.zeros(shape)
        else:
            fan_in = shape[-1] if len(shape) == 2 else HID
            bound = np.sqrt(6.0 / fan_in)
            parts[name] = rng.uniform(-bound, bound, shape)
    return pack(parts)
