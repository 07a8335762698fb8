"""Resident (one cluster per instance) vs tiled schedule: the same arithmetic in the same
order, so every result is bitwise identical; the autotuner's choice cannot change results.
Also parity of the resident schedule with the oracle, and freezing/status under it."""
import numpy as np
import pytest

from gpu_common import compare, lib, oracle_for
from test_gpu_parity import HETERO

pytestmark = pytest.mark.gpu

# mixed precisions, a long instance (17 tiles) and one with Q = 16 in a second batch
MIXED = [dict(d, precision=p) for d, p in zip(HETERO, ("fp64", "fp32", "fp64", "fp32", "fp32+fp64"))]
MIXED.append(dict(nx=530, qx_half=4, qy=4, qz=0, kn=0.2, eta0=0.1, U_left=-0.3, U_right=0.3, grid="tanh",
                  precision="fp32"))
WIDE = [dict(nx=64, qx_half=16, qy=0, qz=0, kn=0.3, eta0=0.1, T_left=0.9, T_right=1.1),
        dict(nx=40, qx_half=12, qy=4, qz=0, kn=0.1, eta0=0.1, U_left=-0.2, U_right=0.2)]


def pair(F, dicts, a, b):
    ps = [F.Params(**d) for d in dicts]
    sa, sb = F.Solver(ps), F.Solver(ps)
    sa.set_schedule(a)
    sb.set_schedule(b)
    return sa, sb


def assert_same(sa, sb):
    ra, sta, na = sa.status()
    rb, stb, nb = sb.status()
    assert np.array_equal(sta, stb) and np.array_equal(na, nb)
    assert np.array_equal(ra, rb, equal_nan=True)
    for i in range(sa.count):
        Ma, Mb = sa.moments(i), sb.moments(i)
        for k in Ma:
            assert np.array_equal(Ma[k], Mb[k], equal_nan=True), (i, k)
        assert sa.get_state(i) == sb.get_state(i), i


@pytest.mark.parametrize("dicts", [MIXED, WIDE], ids=["mixed", "wide"])
def test_resident_equals_tiled_bitwise(dicts):
    F = lib()
    sa, sb = pair(F, dicts, "tiled", "resident")
    assert sb.schedule()[0] == "resident" and sb.schedule()[1] >= 1
    for n in (1, 37, 300):
        sa.step(n)
        sb.step(n)
        assert_same(sa, sb)


def test_resident_freeze_and_status_equal_tiled():
    F = lib()
    dicts = [dict(nx=24, qx_half=4, qy=4, qz=0, kn=0.3, eta0=0.1, U_left=-0.2, U_right=0.2),
             dict(nx=40, qx_half=4, qy=0, qz=0, kn=0.3, eta0=0.1, T_left=0.95, T_right=1.05, precision="fp32+fp64"),
             dict(nx=32, qx_half=4, qy=4, qz=4, kn=0.2, eta0=0.45, U_left=-0.4, U_right=0.4)]   # goes non-finite
    sa, sb = pair(F, dicts, "tiled", "resident")
    for _ in range(20):
        sa.step(500, 2e-6)
        sb.step(500, 2e-6)
    assert_same(sa, sb)
    _, st, _ = sb.status()
    assert st[0] == F.CONVERGED and st[2] == F.FAILED_NONFINITE


def test_resident_matches_oracle():
    F = lib()
    p = F.Params(**HETERO[2])
    s = F.Solver([p])
    s.set_schedule("resident")
    o = oracle_for(p)
    s.step(120)
    o.step(120)
    compare(s.moments(0), o.moments(), 1e-12, "resident schedule")


def test_autotune_picks_a_schedule_without_changing_results():
    F = lib()
    ps = [F.Params(**d) for d in MIXED]
    sa, sb = F.Solver(ps), F.Solver(ps)
    sa.set_schedule("tiled")
    assert sb.schedule()[0] == "auto"
    sb.step(40)                       # shorter than the tuning window: tiled, no choice yet
    assert sb.schedule()[0] == "auto"
    sb.step(200)
    assert sb.schedule()[0] in ("tiled", "resident", "mixed")
    sa.step(240)
    assert_same(sa, sb)
