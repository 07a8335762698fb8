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


def forward_scale(theta, X):
    """Per output, the sum of the magnitudes of the terms of its last-layer sum (bias included),
    with the oracle's BF16-rounded operands: the scale of the FP32 accumulation error."""
    _, (hs, _) = omlp.forward_bf16(theta, X)
    W5, b5 = omlp.unpack(theta)[4]
    return (np.abs(hs[4]) @ np.abs(omlp.bf16(W5)) + np.abs(b5))[:, :3]


def test_forward_matches_oracle():
    """Element-wise against the oracle with BF16 operands where the kernel rounds them.  What
    remains is the FP32 accumulation (~K eps_32 of the sum of |terms| per layer, K <= 128) and,
    rarely, a hidden activation whose FP32 and FP64 values round to neighbouring BF16 numbers
    (one BF16 ulp, 2^-8 relative, of one term).  Each output depends on 4 x 128 rounded
    activations, so a few outputs in a thousand carry such a neighbour (measured 0.6 %).  Bar per
    output: 2e-3 of its scale, and at most 2 % of the outputs beyond 2e-4 of it; a transposed or
    misplaced block errs by O(1) of the scale everywhere."""
    import torch
    F = lib()
    net = F.MLP(max_points=1000, seed=5)
    theta = net.get_params().astype(np.float64)
    assert theta.size == omlp.n_params()
    X = inputs(333, 1)                          # ragged last tile
    y = net.predict(torch.tensor(X, device="cuda")).cpu().numpy()
    ref, _ = omlp.forward_bf16(theta, X.astype(np.float64))
    rel = np.abs(y - ref) / forward_scale(theta, X.astype(np.float64))
    print("forward: max err / scale", rel.max(), "fraction > 2e-4", np.mean(rel > 2e-4))
    assert rel.max() < 2e-3, rel.max()
    assert np.mean(rel > 2e-4) < 2e-2
    # and the plain FP64 network, for scale: BF16 operands cost ~1e-2
    ref64, _ = omlp.forward(theta, X.astype(np.float64))
    assert np.abs(y - ref64).max() / np.abs(ref64).max() < 3e-2


def test_gradient_matches_oracle():
    """Every gradient element against the BF16-operand oracle, relative to the sum of the
    magnitudes of its terms (the FP32 accumulation bound), with the same allowance for rare
    BF16 rounding neighbours as the forward pass.  A transposed or shifted block fails this."""
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
    rl, rg, sc = omlp.loss_and_grad_bf16(theta, X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - rl) < 1e-4 * rl
    g = g.cpu().numpy().astype(np.float64)
    live = sc > 0
    rel = np.abs(g - rg)[live] / sc[live]
    print("gradient: max err / scale", rel.max(), "fraction > 2e-4", np.mean(rel > 2e-4))
    assert rel.max() < 2e-2, rel.max()
    assert np.mean(rel > 2e-4) < 5e-3
    assert np.all(g[~live] == 0.0)
    assert np.all(omlp.unpack(g)[4][0][:, 3:] == 0.0)
    # the FP64 network's gradient, for scale
    _, rg64 = omlp.loss_and_grad(theta, X.astype(np.float64), Y.astype(np.float64))
    assert np.linalg.norm(g - rg64) < 5e-2 * np.linalg.norm(rg64)


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
