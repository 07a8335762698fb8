"""The FP32-storage form over a whole steady-state solve (not just a few hundred steps):
the Couette instance of the sweep (Nx = 200 tanh, 12 x 6 x 4 = 288 velocities, eta0 = 0.1,
Kn = 0.5, u_y = -+0.42) solved to residual 1e-8 with f in FP32, against the same instance in
FP64.  Bar: 1e-5, element-wise, on n and T (relative) and on u_y and Pi_xy (relative to
their largest magnitude).  The channel mass must stay at its initial value."""
import numpy as np
import pytest

from gpu_common import lib

pytestmark = pytest.mark.gpu

KW = dict(nx=200, qx_half=6, qy=6, qz=4, kn=0.5, eta0=0.1, U_left=-0.42, U_right=0.42, grid="tanh", stretch=1.5)


def errors(Ma, Mb):
    return {
        "n": float(np.max(np.abs(Ma["n"] - Mb["n"]) / Mb["n"])),
        "T": float(np.max(np.abs(Ma["T"] - Mb["T"]) / Mb["T"])),
        "uy": float(np.max(np.abs(Ma["uy"] - Mb["uy"])) / np.max(np.abs(Mb["uy"]))),
        "Pxy": float(np.max(np.abs(Ma["Pxy"] - Mb["Pxy"])) / np.max(np.abs(Mb["Pxy"]))),
    }


def cell_widths():
    """x'(s_i) ds of the tanh grid (the oracle's grid: widths only)."""
    from oracle import fdlb as ofd
    o = ofd.Oracle(ofd.Params(nx=KW["nx"], qx_half=1, qy=0, qz=0, kn=0.1, eta0=0.0, grid="tanh", stretch=1.5))
    return o.dx


def test_fp32_solve_matches_fp64_within_1e5():
    F = lib()
    s32 = F.Solver([F.Params(**KW, precision="fp32")])
    s32.run(1e-8, 200000, check_every=500, timeout_s=300.0)
    r32, st32, n32 = s32.status()
    assert st32[0] == F.CONVERGED, (st32, r32)
    M32 = s32.moments(0)
    # FP64 over the same number of steps: the difference is that of the storage precision alone
    s64 = F.Solver([F.Params(**KW, precision="fp64")])
    s64.step(int(n32[0]))
    M64 = s64.moments(0)
    e_same = errors(M32, M64)
    # and FP64 solved to the same residual on its own
    s64b = F.Solver([F.Params(**KW, precision="fp64")])
    s64b.run(1e-8, 200000, check_every=500, timeout_s=300.0)
    e_solve = errors(M32, s64b.moments(0))
    # channel mass sum_i dx_i n_i against the initial uniform state's (n = 1)
    dx = cell_widths()
    m0 = float(np.sum(dx))
    drift32 = abs(float(np.sum(dx * M32["n"])) / m0 - 1.0)
    drift64 = abs(float(np.sum(dx * M64["n"])) / m0 - 1.0)
    print("fp32 vs fp64 at equal steps", e_same, "vs fp64 solve", e_solve, "mass drift fp32/fp64", drift32, drift64,
          "steps", n32, s64b.status()[2])
    assert drift64 < 1e-10
    assert drift32 < 1e-6
    assert all(v <= 1e-5 for v in e_same.values()), e_same
    assert all(v <= 1e-5 for v in e_solve.values()), e_solve
