"""Full-range x quadrature (App. A) on the GPU against the oracle: FP64 at 1e-12 on the three
velocity-space forms, orders 4 to 16 (both widths of the closure kernel's polynomial arrays),
in batches shared with half-range instances; FP32 storage at 1e-5; the resident schedule
bitwise equal to the tiled one."""
import numpy as np
import pytest

from gpu_common import compare, lib, oracle_for
from test_gpu_schedule import assert_same, pair

pytestmark = pytest.mark.gpu

# full-range orders 2 qx_half = 4, 8, 6 (arrays of width 8) and 16 (width 16), ragged node counts
NARROW = [
    dict(nx=40, qx_half=2, qy=0, qz=0, kn=0.2, eta0=0.1, T_left=0.9, T_right=1.1, x_quadrature="full"),
    dict(nx=37, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.15, U_left=-0.3, U_right=0.3, grid="tanh", x_quadrature="full"),
    dict(nx=33, qx_half=3, qy=6, qz=0, kn=0.05, eta0=0.2, U_left=-0.2, U_right=0.42, grid="tanh", j1_shear=True,
         x_quadrature="full"),
    dict(nx=37, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.15, U_left=-0.3, U_right=0.3, grid="tanh"),   # half-range twin
]
WIDE = [
    dict(nx=45, qx_half=8, qy=4, qz=4, kn=0.1, eta0=0.1, accel_y=0.05, x_quadrature="full"),
    dict(nx=50, qx_half=8, qy=0, qz=0, kn=0.5, eta0=0.05, T_left=0.8, T_right=1.2, x_quadrature="full"),
    dict(nx=40, qx_half=6, qy=4, qz=0, kn=0.1, eta0=0.1, accel_y=0.03, grid="tanh"),                  # half-range
]


@pytest.mark.parametrize("steps", [1, 150])
@pytest.mark.parametrize("dicts", [NARROW, WIDE], ids=["narrow", "wide"])
def test_full_range_x_matches_oracle_fp64(dicts, steps):
    F = lib()
    s = F.Solver([F.Params(**d) for d in dicts])
    s.step(steps)
    for i, d in enumerate(dicts):
        o = oracle_for(F.Params(**d))
        o.step(steps)
        compare(s.moments(i), o.moments(), 1e-12, f"instance {i} ({d.get('x_quadrature', 'half')})")
    if dicts is NARROW and steps > 1:
        # the quadrature changes the solution (the full-range twin is not the half-range one)
        assert np.max(np.abs(s.moments(1)["uy"] - s.moments(3)["uy"])) > 1e-6


def test_full_range_x_fp32_storage_within_1e5():
    F = lib()
    d = NARROW[1]
    s = F.Solver([F.Params(**d, precision="fp32")])
    s.step(150)
    o = oracle_for(F.Params(**d))
    o.step(150)
    Mg, Mo = s.moments(0), o.moments()
    for k in ("n", "T"):
        assert np.max(np.abs(Mg[k] - Mo[k]) / Mo[k]) < 1e-5, k
    for k in ("ux", "uy"):
        assert np.max(np.abs(Mg[k] - Mo[k])) < 1e-5, k


def test_full_range_x_resident_equals_tiled():
    F = lib()
    dicts = [dict(d, precision=p) for d, p in zip(NARROW + WIDE[:1], ("fp64", "fp32", "fp64", "fp32", "fp64"))]
    sa, sb = pair(F, dicts, "tiled", "resident")
    for n in (1, 60):
        sa.step(n)
        sb.step(n)
        assert_same(sa, sb)
