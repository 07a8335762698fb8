"""Shared-memory-resident schedule (FDLB_SCHED_MIXED): instances whose three RK buffers fit in
one block's shared memory are stepped by one CTA each, with f kept in shared memory across all
stages and steps of a call; the others take the tiled steps at the same time.  The items are
those of the tiled kernels, so every result is bitwise identical to the tiled schedule's; and
an instance kept in shared memory matches the oracle."""
import numpy as np
import pytest

from gpu_common import compare, lib, oracle_for
from test_gpu_parity import HETERO
from test_gpu_schedule import MIXED, WIDE, assert_same, pair

pytestmark = pytest.mark.gpu

# the bench's Couette instance (200 nodes x 288 velocities, FP32) does not fit: it stays tiled
BIG = dict(nx=200, qx_half=6, qy=6, qz=4, kn=0.5, eta0=0.1, U_left=-0.42, U_right=0.42, grid="tanh", stretch=1.5,
           precision="fp32")


def test_mix_by_size():
    F = lib()
    s = F.Solver([F.Params(**d) for d in MIXED + [BIG]])
    mix = s.schedule_mix()
    prec = [d.get("precision", "fp64") for d in MIXED + [BIG]]
    # three RK buffers + item scratch within one block's shared memory: the 45-node 2D reduced
    # FP32 instance (3 x 144 x 64 x 4 B) and the 70-node 1D reduced one; not the unreduced FP64
    # ones (3 x 128 x 64 x 8 B), the 530-node one (3 x 64 x 544 x 4 B) or the bench instance
    assert mix.tolist() == [0, 1, 0, 1, 0, 0, 0]
    assert prec[4] == "fp32+fp64"                    # the two-phase form stays tiled in any case


# high orders that fit: Q = 16 per side (1D reduced, FP32, 32 nodes) and Q = 12 (1D reduced, FP64)
WIDE_SMALL = [dict(nx=32, qx_half=16, qy=0, qz=0, kn=0.3, eta0=0.1, T_left=0.9, T_right=1.1, precision="fp32"),
              dict(nx=40, qx_half=12, qy=0, qz=0, kn=0.1, eta0=0.1, T_left=1.05, T_right=0.95)] + WIDE


@pytest.mark.parametrize("dicts", [MIXED + [BIG], WIDE_SMALL], ids=["mixed+big", "wide"])
def test_mixed_equals_tiled_bitwise(dicts):
    F = lib()
    sa, sb = pair(F, dicts, "tiled", "mixed")
    assert sb.schedule()[0] == "mixed"
    for n in (1, 37, 300):
        sa.step(n)
        sb.step(n)
        assert_same(sa, sb)


def test_mixed_freeze_and_status_equal_tiled():
    F = lib()
    dicts = [dict(nx=24, qx_half=4, qy=4, qz=0, kn=0.3, eta0=0.1, U_left=-0.2, U_right=0.2),
             dict(nx=40, qx_half=4, qy=0, qz=0, kn=0.3, eta0=0.1, T_left=0.95, T_right=1.05, precision="fp32"),
             dict(nx=32, qx_half=4, qy=4, qz=4, kn=0.2, eta0=0.45, U_left=-0.4, U_right=0.4),   # goes non-finite
             BIG]
    sa, sb = pair(F, dicts, "tiled", "mixed")
    assert sb.schedule_mix()[:3].tolist() == [1, 1, 1]
    for _ in range(20):
        sa.step(500, 2e-6)
        sb.step(500, 2e-6)
    assert_same(sa, sb)
    _, st, _ = sb.status()
    assert st[0] == F.CONVERGED and st[2] == F.FAILED_NONFINITE


def test_smem_resident_matches_oracle():
    F = lib()
    small_poiseuille = dict(nx=24, qx_half=4, qy=4, qz=4, kn=0.05, eta0=0.1, accel_y=0.05, j1_shear=True)
    for d in (small_poiseuille, HETERO[3]):           # unreduced with force and shear term; 1D reduced
        p = F.Params(**d)
        s = F.Solver([p])
        assert s.schedule_mix()[0] == 1
        s.set_schedule("mixed")
        o = oracle_for(p)
        s.step(120)
        o.step(120)
        compare(s.moments(0), o.moments(), 1e-12, "shared-memory-resident schedule")


def test_checkpoint_between_mixed_calls():
    """f returns to global memory at the end of every call: a checkpoint taken between calls
    restarts bitwise."""
    F = lib()
    ps = [F.Params(**HETERO[3])]
    sa, sb = F.Solver(ps), F.Solver(ps)
    assert sa.schedule_mix()[0] == 1
    sa.set_schedule("mixed")
    sb.set_schedule("mixed")
    sa.step(50)
    chk = sa.get_state(0)
    sa.step(50)
    sb.set_state(0, chk)
    sb.step(50)
    assert sa.get_state(0)[8:] == sb.get_state(0)[8:]
    assert np.array_equal(sa.moments(0)["T"], sb.moments(0)["T"])
