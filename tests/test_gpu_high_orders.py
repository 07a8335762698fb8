"""x quadratures beyond 16 per side: the half-range orders of Table 1 (Sec. IV, up to 29 per
side), the orders of the mass-flow runs at large Kn (64, and 100 above Kn = 1, Sec. IV) and
full-range orders beyond 16 (App. A).  The closure's x projections then run in
blocks of 16 orthonormal polynomials (the chain of H products continuing across blocks), the
auxiliary rule grows with the order, and the update loads only its chunk's x-projection rows.
FP64 parity 1e-12 and FP32 1e-5 against the oracle, in one batch with a low-order instance;
tiled and cluster-resident schedules bitwise equal."""
import pytest

from gpu_common import compare, lib, oracle_for
from test_gpu_schedule import assert_same, pair

pytestmark = pytest.mark.gpu

HIGH = [
    dict(nx=40, qx_half=20, qy=0, qz=0, kn=0.3, eta0=0.1, T_left=0.95, T_right=1.05),                  # Fourier, 1D
    dict(nx=36, qx_half=29, qy=0, qz=0, kn=0.5, eta0=0.05, T_left=1.05, T_right=0.95),                 # Table 1's largest
    dict(nx=34, qx_half=20, qy=4, qz=0, kn=0.2, eta0=0.1, U_left=-0.3, U_right=0.3, grid="tanh"),      # Couette, 2D
    dict(nx=40, qx_half=20, qy=0, qz=0, kn=0.3, eta0=0.1, T_left=0.9, T_right=1.1, x_quadrature="full"),   # order 40
    dict(nx=45, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.1, U_left=-0.2, U_right=0.2),                    # low order
]
STEPS = 60


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_high_orders_match_oracle(precision, tol):
    F = lib()
    ps = [F.Params(**d, precision=precision) for d in HIGH]
    s = F.Solver(ps)
    s.set_schedule("tiled")
    s.step(STEPS)
    for i, d in enumerate(HIGH):
        o = oracle_for(F.Params(**d))
        assert abs(s.dt[i] - o.dt) <= 1e-14 * o.dt
        o.step(STEPS)
        compare(s.moments(i), o.moments(), tol, f"instance {i} ({precision})")


def test_high_order_tables_compact():
    """The update block's table holds the x-projection rows of the x-velocities its chunk spans."""
    F = lib()
    s = F.Solver([F.Params(**HIGH[1])])
    chunk, groups, tiles = s.layout(0)
    assert chunk == 16 and groups == (2 * 29 * 2 + 15) // 16


def test_high_orders_resident_equals_tiled_bitwise():
    F = lib()
    sa, sb = pair(F, HIGH, "tiled", "resident")
    for n in (1, 25):
        sa.step(n)
        sb.step(n)
        assert_same(sa, sb)


# Sec. IV's mass-flow orders: 64 per side, and 100 per side above Kn = 1 (Fourier 1D and a
# Poiseuille channel at Kn = 2), with a low-order instance in the same batch
LARGE_KN = [
    dict(nx=30, qx_half=64, qy=0, qz=0, kn=0.5, eta0=0.05, T_left=0.95, T_right=1.05),
    dict(nx=24, qx_half=100, qy=0, qz=0, kn=2.0, eta0=0.02, T_left=1.05, T_right=0.95),
    dict(nx=24, qx_half=100, qy=4, qz=0, kn=2.0, eta0=0.02, accel_y=0.05, flow=2),
    dict(nx=45, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.1, U_left=-0.2, U_right=0.2),
]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_orders_64_and_100_match_oracle(precision, tol):
    F = lib()
    ps = [F.Params(**d, precision=precision) for d in LARGE_KN]
    s = F.Solver(ps)
    s.set_schedule("tiled")
    s.step(20)
    for i, d in enumerate(LARGE_KN):
        o = oracle_for(F.Params(**d))
        assert abs(s.dt[i] - o.dt) <= 1e-14 * o.dt
        o.step(20)
        compare(s.moments(i), o.moments(), tol, f"instance {i} ({precision})")
