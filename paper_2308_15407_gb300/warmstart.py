"""Learned warm start for steady-state solves (no counterpart in the paper).

A small network (``fdlb.MLP``, tcgen05 kernels) maps the channel parameters and a node
position to the steady profiles (n, u_y, T).  A solve then starts from the projected local
equilibrium of the predicted profiles (u_x = 0) instead of the uniform state; the FDLB
iteration itself is unchanged and converges to the same residual.  The predicted density is
rescaled so that the channel holds the same mass as the uniform start (the steady state is
fixed by the mass).

Features (9, zero-padded to 16): flow one-hot (3), log10 Kn + 1, (eta0 - 0.2)/0.2,
Delta T / 0.1 (half the wall temperature difference), U_w / 0.25 - 1 (wall speed),
a_y / 0.05 - 1, 2 x (node position).  Targets: (n - 1)/0.1, u_y/0.5, (T - 1)/0.1.
"""
from __future__ import annotations

import math

import numpy as np

from . import fdlb

NIN = 16


def node_grid(p):
    """Node positions x_i and widths dx_i of the channel [-1/2, 1/2] (cell-centred in s)."""
    N = p.nx
    ds = 2.0 / N
    s = -1.0 + (np.arange(N) + 0.5) * ds
    if p.grid == "uniform":
        return 0.5 * s, np.full(N, 0.5 * ds)
    A = p.stretch
    x = 0.5 * np.tanh(A * s) / math.tanh(A)
    xp = 0.5 * A / (np.cosh(A * s) ** 2 * math.tanh(A))
    return x, xp * ds


def features(p) -> np.ndarray:
    """[nx, 16] float32 network inputs for every node of instance p."""
    x, _ = node_grid(p)
    F = np.zeros((p.nx, NIN), dtype=np.float32)
    F[:, int(p.flow)] = 1.0
    F[:, 3] = math.log10(p.kn) + 1.0
    F[:, 4] = (p.eta0 - 0.2) / 0.2
    F[:, 5] = 0.5 * (p.T_right - p.T_left) / 0.1
    F[:, 6] = 0.5 * (p.U_right - p.U_left) / 0.25 - 1.0
    F[:, 7] = p.accel_y / 0.05 - 1.0
    F[:, 8] = 2.0 * x
    return F


def targets(M) -> np.ndarray:
    return np.stack([(M["n"] - 1.0) / 0.1, M["uy"] / 0.5, (M["T"] - 1.0) / 0.1], axis=1).astype(np.float32)


def profiles(pred: np.ndarray, p):
    """Network outputs -> (n, u_y, T) with n rescaled to unit mass and T kept positive."""
    n = 1.0 + 0.1 * pred[:, 0].astype(np.float64)
    uy = 0.5 * pred[:, 1].astype(np.float64)
    T = 1.0 + 0.1 * pred[:, 2].astype(np.float64)
    n = np.maximum(n, 0.2)
    T = np.maximum(T, 0.2)
    _, dx = node_grid(p)
    n *= 1.0 / float(np.sum(dx * n))
    if p.qy == 0:
        uy = np.zeros_like(uy)
    return n, uy, T


class WarmStart:
    """Training set from solved instances, the network, and initial profiles for new ones."""

    def __init__(self, max_points: int, seed: int = 1, device="cuda"):
        self.net = fdlb.MLP(max_points=max_points, seed=seed, device=device)
        self.device = device

    @staticmethod
    def dataset(solver, converged_only=True):
        """(X, Y) from the current state of every (converged) instance of a Solver."""
        _, st, _ = solver.status()
        X, Y = [], []
        for i, p in enumerate(solver.params):
            if converged_only and st[i] != fdlb.CONVERGED:
                continue
            X.append(features(p))
            Y.append(targets(solver.moments(i)))
        return np.concatenate(X), np.concatenate(Y)

    def fit(self, X, Y, steps=2000, lr=3e-3, lr_min=1e-4):
        """Full-batch Adam with a cosine-decayed learning rate; returns the loss history."""
        import torch
        xd = torch.tensor(X, device=self.device)
        yd = torch.tensor(Y, device=self.device)
        hist = []
        for k in range(steps):
            rate = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * k / steps))
            loss, _ = self.net.train_step(xd, yd, rate)
            if k % 100 == 0 or k == steps - 1:
                hist.append(loss)
        return hist

    def apply(self, solver, insts=None):
        """Reset the given instances (default all) to the predicted local equilibrium."""
        import torch
        insts = range(solver.count) if insts is None else insts
        for i in insts:
            p = solver.params[i]
            pred = self.net.predict(torch.tensor(features(p), device=self.device)).cpu().numpy()
            n, uy, T = profiles(pred, p)
            solver.set_profiles(i, n, uy, T)
