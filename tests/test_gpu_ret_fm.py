"""Fischer-Methfessel contact value (Eq. chi_ret) on the GPU against the oracle: FP64 at
1e-12, FP32 storage at 1e-5, mixed with SET instances in one batch, both grids."""
import numpy as np
import pytest

from gpu_common import compare, lib, oracle_for

pytestmark = pytest.mark.gpu

# sigma = 6 sqrt(2) eta0 chi(eta0) Kn: 0.055 (uniform, +-3.5 cells) and 0.041 (tanh)
FM = [
    dict(nx=64, qx_half=4, qy=0, qz=0, kn=0.05, eta0=0.1, T_left=0.95, T_right=1.05, chi_model="ret-fm"),
    dict(nx=45, qx_half=6, qy=4, qz=0, kn=0.02, eta0=0.2, U_left=-0.3, U_right=0.3, grid="tanh", chi_model="ret-fm"),
    dict(nx=40, qx_half=4, qy=4, qz=4, kn=0.03, eta0=0.15, accel_y=0.05, chi_model="ret-fm"),
]


@pytest.mark.parametrize("steps", [1, 120])
def test_ret_fm_matches_oracle_fp64(steps):
    F = lib()
    dicts = FM + [{**FM[0], "chi_model": "set"}]
    s = F.Solver([F.Params(**d) for d in dicts])
    s.step(steps)
    for i, d in enumerate(dicts):
        o = oracle_for(F.Params(**d))
        o.step(steps)
        compare(s.moments(i), o.moments(), 1e-12, f"instance {i} ({d['chi_model']})")
    if steps > 1:
        # the averaged contact value changes the solution (not accidentally the SET one)
        assert np.max(np.abs(s.moments(0)["n"] - s.moments(3)["n"])) > 1e-9


def test_ret_fm_fp32_storage_within_1e5():
    F = lib()
    p = F.Params(**{**FM[1], "precision": "fp32"})
    s = F.Solver([p])
    s.step(120)
    o = oracle_for(F.Params(**FM[1]))
    o.step(120)
    Mg, Mo = s.moments(0), o.moments()
    for k in ("n", "T"):
        assert np.max(np.abs(Mg[k] - Mo[k]) / Mo[k]) < 1e-5, k
    for k in ("ux", "uy"):
        assert np.max(np.abs(Mg[k] - Mo[k])) < 1e-5, k
