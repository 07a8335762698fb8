"""Seeded workload generators (no GPU): the same seed gives the same instances, every draw
stays in its documented range, each flow uses only its own driving parameter, and every
instance passes the library's parameter validation."""
import numpy as np

from paper_2308_15407_gb300 import fdlb as F
from paper_2308_15407_gb300 import workloads as W


def test_batched_sweep_is_seeded_and_in_range():
    a, b = W.batched_sweep(256), W.batched_sweep(256)
    assert a == b
    assert a != W.batched_sweep(256, seed=1)
    flows = set()
    for d in a:
        flows.add(d["flow"])
        assert 32 <= d["nx"] <= 512 and d["qx_half"] in (4, 6, 8)
        assert 0.01 <= d["kn"] <= 1.0 and 0.01 <= d["eta0"] <= 0.45
        if d["flow"] == W.FOURIER:
            assert d["qy"] == 0 and abs(d["T_left"] + d["T_right"] - 2.0) < 1e-12
            assert 0.8 <= d["T_left"] <= 1.0
        elif d["flow"] == W.COUETTE:
            assert d["qy"] == 4 and d["U_left"] == -d["U_right"] and 0 <= d["U_right"] <= 0.5
            assert "accel_y" not in d
        else:
            assert d["qy"] == 4 and 0 <= d["accel_y"] <= 0.1 and "U_left" not in d
    assert flows == {W.FOURIER, W.COUETTE, W.POISEUILLE}


def test_generated_instances_pass_validation():
    sets = [W.batched_sweep(64), W.couette_sweep(), W.fourier_5000(), W.couette_family(8, seed=5),
            [W.paper_geometry(4, 0.1), W.paper_geometry(10, 0.01, flow="couette", U_w=1.0, cells_per_sigma=20)],
            W.knudsen_sweep(R_values=(2, 20), points=3)[0]]
    for dicts in sets:
        assert F.workspace_bytes([F.Params(**d) for d in dicts]) > 0


def test_couette_family_ranges():
    fam = W.couette_family(50, seed=23085)
    assert fam == W.couette_family(50, seed=23085)
    e = np.array([d["eta0"] for d in fam])
    kn = np.log10([d["kn"] for d in fam])
    u = np.array([d["U_right"] for d in fam])
    assert e.min() >= 0.05 and e.max() <= 0.25
    assert kn.min() >= -1.5 and kn.max() <= -0.3
    assert u.min() >= 0.3 and u.max() <= 0.5
