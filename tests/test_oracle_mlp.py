"""Pins of the picker-MLP oracle: finite differences, closed forms, Adam."""
import numpy as np

from oracle import mlp as M


def _data(n=17, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, M.IN)), rng.uniform(0, 1, n)


def test_parameter_count():
    assert M.NPARAM == 128 * 66 + 128 + 128 * 128 + 128 + 128 + 1


def test_gradient_matches_central_differences():
    X, t = _data()
    theta = M.init(3) * 0.5
    theta[-1] = 0.1
    _, g = M.loss_and_grad(theta, X, t)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(M.NPARAM, 60, replace=False), [M.NPARAM - 1]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss(tp, X, t) - M.loss(tm, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_network_outputs_bias_and_its_gradient():
    X, t = _data()
    theta = np.zeros(M.NPARAM)
    theta[-1] = 0.25
    y, _ = M.forward(theta, X)
    assert np.all(y == 0.25)
    loss, g = M.loss_and_grad(theta, X, t)
    assert abs(loss - np.mean((0.25 - t) ** 2)) < 1e-15
    assert abs(g[-1] - 2 * np.mean(0.25 - t)) < 1e-15
    assert np.all(g[:-1] == 0.0)           # every ReLU is off: no other gradient


def test_hand_computed_forward():
    # one active path: x0 -> h1[0] (weight 2, bias 1) -> h2[0] (weight 3) -> y (weight 0.5, bias -1)
    theta = np.zeros(M.NPARAM)
    p = M.unpack(theta)
    p["W1"][0, 0] = 2.0
    p["b1"][0] = 1.0
    p["W2"][0, 0] = 3.0
    p["w3"][0] = 0.5
    p["b3"][0] = -1.0
    theta = M.pack(p)
    X = np.zeros((3, M.IN))
    X[:, 0] = [1.0, -0.25, -2.0]
    y, _ = M.forward(theta, X)
    # h1 = relu(2x+1) = 3, 0.5, 0 ; h2 = 3 h1 ; y = 0.5 h2 - 1
    assert np.allclose(y, [3.5, -0.25, -1.0], rtol=0, atol=1e-15)


def test_adam_first_step_is_a_signed_lr_step():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    theta = np.ones(4)
    new, m, v = M.adam(theta, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2, update lr g / (|g| + eps)
    assert np.allclose(new, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.all(np.abs(new[:3] - theta[:3]) <= 0.01)


def test_training_reduces_loss():
    X, t = _data(64, 2)
    theta = M.init(0)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    l0, _ = M.loss_and_grad(theta, X, t)
    for step in range(1, 201):
        _, g = M.loss_and_grad(theta, X, t)
        theta, m, v = M.adam(theta, g, m, v, step)
    assert M.loss(theta, X, t) < 0.1 * l0


def test_soft_level_loss_derivative_and_limits():
    rng = np.random.default_rng(8)
    L = rng.uniform(0, 0.3, (9, 64))
    L[np.arange(9), rng.integers(0, 64, 9)] = 0.0
    y = rng.uniform(0.05, 0.95, 9)
    for sigma in (0.7, 1.5, 4.0):
        v, dv = M.soft_level_loss(y, L, sigma)
        h = 1e-6
        vp, _ = M.soft_level_loss(y + h, L, sigma)
        vm, _ = M.soft_level_loss(y - h, L, sigma)
        np.testing.assert_allclose(dv, (vp - vm) / (2 * h), rtol=1e-5, atol=1e-7)
        assert (v >= L.min(axis=1) - 1e-12).all() and (v <= L.max(axis=1) + 1e-12).all()
    # a narrow window sits on the nearest level: the ARI lost there
    v, _ = M.soft_level_loss(np.array([10 / 64, 33.2 / 64]), L[:2], 0.05)
    np.testing.assert_allclose(v, [L[0, 9], L[1, 32]], rtol=1e-9, atol=1e-12)
    # a flat table has no slope
    _, dv = M.soft_level_loss(y, np.full((9, 64), 0.1), 1.0)
    np.testing.assert_allclose(dv, 0.0, atol=1e-9)


def test_mixed_loss_gradient_matches_central_differences():
    X, t = _data(13, seed=4)
    L = np.random.default_rng(5).uniform(0, 0.2, (13, 64))
    theta = M.init(6)
    theta[-1] = 0.4
    for mix in (0.0, 0.3, 1.0):
        lo, g = M.mixed_loss_and_grad(theta, X, t, L, 1.5, mix)
        if mix == 1.0:
            lm, gm = M.loss_and_grad(theta, X, t)
            assert abs(lo - lm) < 1e-12 and np.allclose(g, gm)
        rng = np.random.default_rng(int(mix * 10))
        for k in rng.choice(M.NPARAM, 12, replace=False):
            e = np.zeros(M.NPARAM)
            e[k] = 1e-6
            fp, _ = M.mixed_loss_and_grad(theta + e, X, t, L, 1.5, mix)
            fm, _ = M.mixed_loss_and_grad(theta - e, X, t, L, 1.5, mix)
            assert abs((fp - fm) / 2e-6 - g[k]) <= 1e-6 + 1e-4 * abs(g[k])
