"""Pins of the FP64 surrogate-network oracle: finite differences of the loss, the BCE value
and slope at known points, and the closed form of Adam's first step."""
import math

import numpy as np

from oracle import mlp


def _net(d=5, w=7, seed=0):
    g = np.random.default_rng(seed)
    n = sum(int(np.prod(s)) for s in mlp.shapes(d, w))
    theta = g.standard_normal(n) * 0.5
    X = g.standard_normal((13, d))
    y = (g.random(13) < 0.5).astype(float)
    return theta, X, y, d, w


def test_backprop_matches_central_differences():
    theta, X, y, d, w = _net()
    _, g = mlp.loss_and_grad(theta, X, y, d, w)
    h = 1e-6
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, y, d, w)[0] - mlp.loss_and_grad(tm, X, y, d, w)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 + 1e-5 * abs(g[i]), i


def test_bce_values():
    assert abs(mlp.bce([0.0], [1.0]) - math.log(2)) < 1e-15
    assert abs(mlp.bce([0.0], [0.0]) - math.log(2)) < 1e-15
    assert mlp.bce([50.0], [1.0]) < 1e-20 and abs(mlp.bce([50.0], [0.0]) - 50.0) < 1e-12


def test_logit_gradient_is_sigmoid_minus_label():
    d, w = 3, 4
    theta = np.zeros(sum(int(np.prod(s)) for s in mlp.shapes(d, w)))
    theta[-1] = 0.7  # b4: z = 0.7 for every sample
    X = np.ones((4, d))
    y = np.array([1.0, 0.0, 1.0, 1.0])
    _, g = mlp.loss_and_grad(theta, X, y, d, w)
    s = 1 / (1 + math.exp(-0.7))
    assert abs(g[-1] - np.mean(s - y)) < 1e-15


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
