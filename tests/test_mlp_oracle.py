"""Pins of the float64 proposal-network reference (oracle/mlp.py).

The network is not part of the paper; its reference is pinned by closed forms
(zero weights, a hand-built one-path network, Adam's first step), central
finite differences of the loss, and invariants of the feature map.
"""
import numpy as np

from oracle import mlp


def test_param_count():
    assert mlp.N_PARAMS == 8 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4801


def test_zero_weights_give_bias():
    p = np.zeros(mlp.N_PARAMS)
    p[-1] = 1.25
    X = np.random.default_rng(0).normal(size=(7, 8))
    assert np.all(mlp.forward(p, X) == 1.25)


def test_hand_built_path():
    # out = 3 * relu(2 * relu(x0 - 1) + 0.5) + 0.1, through unit 5 of h1 and unit 9 of h2
    d = mlp.unpack(np.zeros(mlp.N_PARAMS))
    d = {k: v.copy() for k, v in d.items()}
    d["W1"][0, 5] = 1.0
    d["b1"][5] = -1.0
    d["W2"][5, 9] = 2.0
    d["b2"][9] = 0.5
    d["W3"][9] = 3.0
    d["b3"][0] = 0.1
    p = mlp.pack(d)
    X = np.zeros((4, 8))
    X[:, 0] = [0.0, 1.0, 2.0, 4.0]
    expect = 3 * np.maximum(2 * np.maximum(X[:, 0] - 1, 0) + 0.5, 0) + 0.1
    np.testing.assert_allclose(mlp.forward(p, X), expect, rtol=0, atol=1e-15)
    assert abs(mlp.loss(p, X, expect)) < 1e-28
    assert np.all(mlp.grad(p, X, expect) == 0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(5)
    X = rng.normal(size=(16, 8))
    y = rng.normal(size=16)
    g = mlp.grad(p, X, y)
    idx = rng.choice(mlp.N_PARAMS, size=120, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, 0, 512, 576, 4672]])  # each block touched
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, y) - mlp.loss(p - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_first_step_closed_form():
    # t = 1: m_hat = g, v_hat = g^2, so the step is -lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 1.0, 1.0, 1.0])
    p1, m, v = mlp.adam_step(p, g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_feature_invariants():
    f = mlp.features(deg=[3, 0, 10], dS=[2, 1, 4], ub=[100, -1, 0], stamp=[1, 4, 2], two_hop=[7, 0, 1],
                     mx=[3, 1, 4], rnd=4, prev_gain=50)
    np.testing.assert_allclose(f[:, 0], np.log1p([3, 0, 10]))
    assert list(f[:, 1]) == [2, 1, 4]
    assert f[1, 2] == 0 and f[2, 2] == 0           # bounds below zero count as 0
    assert list(f[:, 3]) == [3, 0, 2]               # rounds since the last evaluation
    assert list(f[:, 5]) == [1, 0, 0]               # mx - d_S
    assert np.all(f[:, 6] == np.log1p(50))
    np.testing.assert_allclose(f[:, 7], f[:, 2] - f[:, 6])
