"""Warm-start network kernels (tcgen05, BF16 operands, FP32 accumulation) against the FP64
oracle of oracle/mlp.py on the same weights: forward values, backprop gradient, and a
training run that lowers the loss."""
import numpy as np
import pytest

from gpu_common import lib
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def inputs(P, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((P, 16), dtype=np.float32)
    X[:, :9] = rng.uniform(-1, 1, (P, 9))
    return X


def test_forward_matches_oracle():
    import torch
    F = lib()
    net = F.MLP(max_points=1000, seed=5)
    theta = net.get_params().astype(np.float64)
    assert theta.size == omlp.n_params()
    X = inputs(333, 1)                          # ragged last tile
    y = net.predict(torch.tensor(X, device="cuda")).cpu().numpy()
    ref, _ = omlp.forward(theta, X.astype(np.float64))
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err < 3e-2, err                      # BF16 operands, FP32 accumulation


def test_gradient_matches_oracle():
    import torch
    F = lib()
    net = F.MLP(max_points=512, seed=9)
    rng = np.random.default_rng(2)
    theta = (net.get_params().astype(np.float64) + rng.normal(0, 0.02, omlp.n_params()))
    layers = omlp.unpack(theta)
    layers[4][0][:, 3:] = 0.0                   # unused output columns stay zero
    net.set_params(theta.astype(np.float32))
    theta = net.get_params().astype(np.float64)
    X = inputs(300, 3)
    Y = rng.normal(0, 0.5, (300, 3)).astype(np.float32)
    loss, g = net.train_step(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), lr=0.0, want_grad=True)
    rl, rg = omlp.loss_and_grad(theta, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - rl) < 2e-2 * rl
    g = g.cpu().numpy().astype(np.float64)
    cos = g @ rg / (np.linalg.norm(g) * np.linalg.norm(rg))
    rel = np.linalg.norm(g - rg) / np.linalg.norm(rg)
    assert cos > 0.999 and rel < 5e-2, (cos, rel)
    # per layer as well
    for (gw, gb), (rw, rb) in zip(omlp.unpack(g), omlp.unpack(rg)):
        assert np.linalg.norm(gw - rw) <= 6e-2 * np.linalg.norm(rw) + 1e-9
    assert np.all(omlp.unpack(g)[4][0][:, 3:] == 0.0)


def test_training_lowers_the_loss():
    import torch
    F = lib()
    P = 4096
    net = F.MLP(max_points=P, seed=1)
    X = inputs(P, 4)
    Y = np.stack([np.sin(2 * X[:, 0]) * X[:, 1], 0.5 * X[:, 2] ** 2 - X[:, 3], np.tanh(X[:, 4] + X[:, 5])], axis=1).astype(np.float32)
    xd, yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    first, _ = net.train_step(xd, yd, lr=3e-3)
    for _ in range(300):
        last, _ = net.train_step(xd, yd, lr=3e-3)
    assert last < 0.1 * first, (first, last)
