"""Pins of the warm-start network oracle: GELU closed forms, backprop gradient against
central finite differences of the loss, one Adam step written out by hand."""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_forms():
    z = np.array([0.0, 1.0, -1.0, 8.0, -8.0])
    g = mlp.gelu(z)
    assert g[0] == 0.0
    assert abs(g[1] - 0.8413447460685429) < 1e-15            # Phi(1)
    assert abs(g[2] + 0.15865525393145707) < 1e-15           # -Phi(-1)
    assert abs(g[3] - 8.0) < 1e-13 and abs(g[4]) < 1e-13
    # derivative against a central difference
    for x in (-2.0, -0.3, 0.0, 0.7, 1.9):
        h = 1e-6
        fd = (mlp.gelu(np.array([x + h])) - mlp.gelu(np.array([x - h])))[0] / (2 * h)
        assert abs(mlp.gelu_grad(np.array([x]))[0] - fd) < 1e-8


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    n = mlp.n_params()
    theta = rng.normal(0, 0.15, n)
    X = np.zeros((6, 16))
    X[:, :9] = rng.normal(0, 1, (6, 9))
    Y = rng.normal(0, 0.5, (6, 3))
    loss, g = mlp.loss_and_grad(theta, X, Y)
    idx = rng.choice(n, 40, replace=False)
    # include parameters of every layer, and the unused output columns (gradient exactly 0)
    layers = mlp.unpack(np.arange(n, dtype=float))
    idx = np.concatenate([idx, [int(layers[0][0][0, 0]), int(layers[4][0][5, 2]), int(layers[4][1][2]), int(layers[4][0][3, 10])]])
    h = 1e-6
    for j in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (mlp.loss_and_grad(tp, X, Y)[0] - mlp.loss_and_grad(tm, X, Y)[0]) / (2 * h)
        assert abs(g[j] - fd) < 1e-7 + 1e-5 * abs(fd), (j, g[j], fd)
    assert g[int(layers[4][0][3, 10])] == 0.0


def test_adam_step_by_hand():
    th = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    new, m, v = mlp.adam_step(th, np.zeros(2), np.zeros(2), g, 1, 0.01)
    # t = 1: m_hat = g, v_hat = g^2, step = lr * g / (|g| + eps)
    np.testing.assert_allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
