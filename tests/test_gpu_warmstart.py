"""Learned warm start: a network trained on steady states the solver produced predicts the
profiles of fresh instances; started there, the unchanged FDLB iteration reaches the same
residual in fewer steps and the same steady state."""
import numpy as np
import pytest

from gpu_common import lib
from paper_2308_15407_gb300 import workloads

pytestmark = pytest.mark.gpu

KW = dict(nx=40, qx_half=4, qy=4, qz=0, grid="uniform", precision="fp64")


def solve(F, dicts, warm=None, require_all=True):
    s = F.Solver([F.Params(**d) for d in dicts])
    if warm is not None:
        warm.apply(s)
    s.run(1e-8, 200000, check_every=1000)
    r, st, ns = s.status()
    if require_all:
        assert np.all(st == F.CONVERGED)
    return s, ns


def test_warm_start_reaches_same_state_in_fewer_steps():
    F = lib()
    from paper_2308_15407_gb300.warmstart import WarmStart
    train = workloads.couette_family(48, seed=11, **KW)
    s_train, _ = solve(F, train, require_all=False)
    X, Y = WarmStart.dataset(s_train)
    ws = WarmStart(max_points=X.shape[0], seed=3)
    hist = ws.fit(X, Y, steps=1500)
    assert hist[-1] < 0.05 * hist[0]
    test = workloads.couette_family(16, seed=12, **KW)
    cold, n_cold = solve(F, test)
    warm, n_warm = solve(F, test, warm=ws)
    # steps scale with the logarithm of the initial error: profiles accurate to ~1 % save ~20 %
    assert np.mean(n_warm) < 0.9 * np.mean(n_cold), (np.mean(n_warm), np.mean(n_cold))
    for i in range(len(test)):
        Mc, Mw = cold.moments(i), warm.moments(i)
        for k in ("n", "T", "uy"):
            assert np.max(np.abs(Mc[k] - Mw[k])) < 2e-4, (i, k)
