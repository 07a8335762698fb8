"""The 2048-instance mixed sweep (uneven nodes and orders, all flows, reduced velocity sets)
in one batch: sampled instances against the oracle, and the status of every instance."""
import numpy as np
import pytest

from gpu_common import lib, oracle_for
from paper_2308_15407_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_batched_sweep_sampled_parity_fp32():
    F = lib()
    dicts = workloads.batched_sweep()
    params = [F.Params(**d) for d in dicts]
    s = F.Solver(params)
    steps = 40
    s.step(steps)
    r, st, ns = s.status()
    # every instance either advanced all steps or was stopped by the status logic
    assert set(np.unique(st)).issubset({F.ACTIVE, F.FAILED_NONFINITE, F.FAILED_UNPHYSICAL})
    assert np.all(ns[st == F.ACTIVE] == steps)
    # sampled stable instances (eta0 <= 0.2), one per flow, plus the largest node count
    rng = np.random.Generator(np.random.PCG64(7))
    stable = [i for i, d in enumerate(dicts) if d["eta0"] <= 0.2 and st[i] == F.ACTIVE]
    picks = []
    for flow in (0, 1, 2):
        cand = [i for i in stable if dicts[i]["flow"] == flow]
        picks.append(int(rng.choice(cand)))
    picks.append(max(stable, key=lambda i: dicts[i]["nx"]))
    for i in picks:
        o = oracle_for(F.Params(**{**dicts[i], "precision": "fp64"}))
        o.step(steps)
        Mg, Mo = s.moments(i), o.moments()
        for k in ("n", "T"):
            assert np.max(np.abs(Mg[k] - Mo[k]) / Mo[k]) < 1e-5, (i, dicts[i], k)
        for k in ("ux", "uy"):
            assert np.max(np.abs(Mg[k] - Mo[k])) < 1e-5, (i, dicts[i], k)
