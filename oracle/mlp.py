"""FP64 CPU oracle of the warm-start network (test infrastructure only, see oracle/__init__).

The network predicts the steady profiles (n, u_y, T) at a grid node from the channel
parameters and the node position: 16 inputs (9 features, zero-padded), 4 hidden layers of
128 units with the exact GELU activation, 16 outputs of which the first 3 are used.
Layer l computes z_l = h_{l-1} W_l + b_l with W_l stored [inputs x outputs].
Loss: mean squared error over the points and the 3 used outputs.  Optimiser: Adam.

This part has no counterpart in the paper (it is a learned initial guess for the FDLB
iteration).  Pins: the gradient against central finite differences of the loss, closed-form
GELU values, and one Adam step against the update written out by hand.
"""
from __future__ import annotations

import math

import numpy as np

SIZES = [16, 128, 128, 128, 128, 16]
NOUT = 3


def _erf(x):
    return np.vectorize(math.erf, otypes=[float])(x)


def gelu(z):
    """z * Phi(z) with Phi the standard normal CDF."""
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def n_params():
    return sum(SIZES[l] * SIZES[l + 1] + SIZES[l + 1] for l in range(5))


def unpack(theta):
    """Flat parameter vector -> [(W_l, b_l)] in the order W1, b1, ..., W5, b5."""
    out, o = [], 0
    for l in range(5):
        a, b = SIZES[l], SIZES[l + 1]
        W = theta[o:o + a * b].reshape(a, b)
        o += a * b
        bb = theta[o:o + b]
        o += b
        out.append((W, bb))
    return out


def forward(theta, X):
    """Returns (prediction [P, 3], cache of pre-activations and activations)."""
    layers = unpack(np.asarray(theta, dtype=np.float64))
    h = np.asarray(X, dtype=np.float64)
    hs, zs = [h], []
    for l, (W, b) in enumerate(layers):
        z = h @ W + b
        zs.append(z)
        h = gelu(z) if l < 4 else z
        hs.append(h)
    return h[:, :NOUT], (hs, zs)


def loss_and_grad(theta, X, Y):
    """MSE loss (1/(3P)) sum (pred - Y)^2 and its gradient with respect to theta (backprop)."""
    layers = unpack(np.asarray(theta, dtype=np.float64))
    pred, (hs, zs) = forward(theta, X)
    P = X.shape[0]
    diff = pred - Y
    loss = float(np.sum(diff * diff) / (NOUT * P))
    d = np.zeros_like(zs[-1])
    d[:, :NOUT] = 2.0 * diff / (NOUT * P)
    grads = [None] * 5
    for l in range(4, -1, -1):
        W, _ = layers[l]
        gW = hs[l].T @ d
        gb = d.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            d = (d @ W.T) * gelu_grad(zs[l - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1): returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ----------------------------------------------------------------------------
# The same network with the GEMM operands rounded to BF16 where the tensor-core kernels round
# them (FP32 value -> BF16, round to nearest even), everything else in FP64.  Used for
# element-wise checks of the kernels: the remaining difference is the FP32 accumulation order
# and, rarely, an operand whose FP32 and FP64 values round to neighbouring BF16 numbers.
# ----------------------------------------------------------------------------

def bf16(x):
    """Round to the nearest BF16 (ties to even) through the FP32 value, returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, X, rnd=bf16):
    """Forward pass with BF16 operands: the inputs, every weight matrix and every hidden
    activation GELU(z) enter their GEMM rounded; biases and pre-activations stay exact.
    Returns (prediction [P, 3], cache (rounded activations, pre-activations))."""
    layers = unpack(np.asarray(theta, dtype=np.float64))
    h = rnd(X)
    hs, zs = [h], []
    for l, (W, b) in enumerate(layers):
        z = h @ rnd(W) + b
        zs.append(z)
        h = rnd(gelu(z)) if l < 4 else z
        hs.append(h)
    return h[:, :NOUT], (hs, zs)


def loss_and_grad_bf16(theta, X, Y, rnd=bf16):
    """Backprop with the operands of every GEMM rounded as in the kernels: dW_l = H_{l-1}^T dZ_l
    with both factors rounded, dH_{l-1} = dZ_l W_l^T with both rounded, db_l = column sums of the
    rounded dZ_l.  Also returns, per parameter, the sum of the magnitudes of the terms of its
    sum (the scale of the FP32 accumulation error)."""
    layers = unpack(np.asarray(theta, dtype=np.float64))
    pred, (hs, zs) = forward_bf16(theta, X, rnd)
    P = X.shape[0]
    diff = pred - Y
    loss = float(np.sum(diff * diff) / (NOUT * P))
    d = np.zeros_like(zs[-1])
    d[:, :NOUT] = 2.0 * diff / (NOUT * P)
    grads, scales = [None] * 5, [None] * 5
    for l in range(4, -1, -1):
        W, _ = layers[l]
        dr = rnd(d)
        gW = hs[l].T @ dr
        gb = dr.sum(axis=0)
        grads[l] = (gW, gb)
        scales[l] = (np.abs(hs[l]).T @ np.abs(dr), np.abs(dr).sum(axis=0))
        if l > 0:
            d = (dr @ rnd(W).T) * gelu_grad(zs[l - 1])
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    scale = np.concatenate([np.concatenate([sW.ravel(), sb]) for sW, sb in scales])
    return loss, flat, scale
