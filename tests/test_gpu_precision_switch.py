"""FP32-then-FP64 precision form: the switch on stagnation, the exact up-cast of f, the FP64
continuation against the oracle, checkpoints across the switch, and the solve to a tolerance
below the FP32 residual floor."""
import numpy as np
import pytest

from gpu_common import compare, lib, oracle_for

pytestmark = pytest.mark.gpu

# Fourier, 1D reduced velocity set (16 velocities): FP32 storage stalls far above 1e-11
KW = dict(nx=40, qx_half=4, qy=0, qz=0, kn=0.3, eta0=0.1, T_left=0.95, T_right=1.05)
WINDOW = 2000


def state_f(F, s, inst, p):
    """f of instance inst from its checkpoint, as an array [2Q, Tc, nx] (oracle layout)."""
    st = s.get_state(inst)
    pr, _ = s.precision_state()
    two_phase = p.precision == "fp32+fp64"
    off = 24 + (16 if two_phase else 0)
    dtype = np.float64 if pr[inst] == F.FP64 else np.float32
    ld = (p.nx + 31) // 32 * 32
    K = s.nvel[inst]
    f = np.frombuffer(st, dtype=dtype, offset=off, count=K * ld)
    return f.reshape(2 * p.qx_half, K // (2 * p.qx_half), ld)[:, :, :p.nx].astype(np.float64), st


def test_switch_is_exact_upcast_then_fp64_parity():
    F = lib()
    ps = [F.Params(**KW, precision=x) for x in ("fp32", "fp32+fp64", "fp64")]
    s = F.Solver(ps)
    pr, sw = s.precision_state()
    assert pr.tolist() == [F.FP32_STORAGE, F.FP32_STORAGE, F.FP64] and sw.tolist() == [-1, -1, -1]
    # the state layout used below: the FP64 instance's initial f is the oracle's
    o = oracle_for(ps[2])
    f64, _ = state_f(F, s, 2, ps[2])
    np.testing.assert_allclose(f64, o.f, rtol=1e-13, atol=1e-16)
    dx = np.full(KW["nx"], 1.0 / KW["nx"])
    mass0 = float(np.sum(dx * s.moments(1)["n"]))
    # step one at a time until the two-phase instance switches; the plain FP32 instance runs
    # the same float arithmetic, so at the switch its f is the two-phase f before the up-cast
    S = None
    for k in range(1, 3 * WINDOW):
        s.step(1)
        pr, sw = s.precision_state()
        if pr[1] == F.FP64:
            S = k
            break
    assert S is not None, "no switch within three stagnation windows"
    assert sw[1] == S and pr[0] == F.FP32_STORAGE
    f32, _ = state_f(F, s, 0, ps[0])
    fup, _ = state_f(F, s, 1, ps[1])
    # up-cast times one factor that restores the mass of the anchor
    c = fup / f32
    assert np.all(np.abs(c / c.flat[0] - 1.0) < 4e-16), "up-cast is not one uniform factor"
    m32 = float(np.sum(dx * s.moments(0)["n"]))
    assert abs(c.flat[0] * m32 / mass0 - 1.0) < 1e-13
    assert abs(np.sum(dx * s.moments(1)["n"]) / mass0 - 1.0) < 1e-14
    assert s.status()[2][1] == S
    # one FP64 step (its first-stage moments are the rescaled FP32 ones), then parity with the oracle
    # started from the two-phase f
    s.step(1)
    f1, chk = state_f(F, s, 1, ps[1])
    o = oracle_for(F.Params(**KW, precision="fp64"))
    o.f = f1.copy()
    s.step(30)
    o.step(30)
    compare(s.moments(1), o.moments(), 1e-12, "FP64 phase after the up-cast")
    # a checkpoint keeps the phase; set_profiles restarts the FP32 phase
    x = np.linspace(-0.5, 0.5, KW["nx"])
    s.set_profiles(1, np.ones_like(x), np.zeros_like(x), 1.0 + 0.05 * x)
    pr, sw = s.precision_state()
    assert pr[1] == F.FP32_STORAGE and sw[1] == -1
    s.set_state(1, chk)
    pr, sw = s.precision_state()
    assert pr[1] == F.FP64 and sw[1] == S
    assert s.status()[2][1] == S + 1
    assert s.get_state(1) == chk


def test_two_phase_solve_below_fp32_floor():
    F = lib()
    ps = [F.Params(**KW, precision=x) for x in ("fp32+fp64", "fp32", "fp64")]
    s = F.Solver(ps)
    tol = 1e-11
    for _ in range(60):
        s.step(2000, tol)
        r, st, ns = s.status()
        if st[0] != F.ACTIVE and st[2] != F.ACTIVE:
            break
    r, st, ns = s.status()
    pr, sw = s.precision_state()
    assert st[2] == F.CONVERGED and r[2] < tol
    assert st[0] == F.CONVERGED and r[0] < tol, (r, st, ns)
    assert pr[0] == F.FP64 and 0 < sw[0] < ns[0]
    # plain FP32 storage cannot resolve a residual this small
    assert st[1] != F.CONVERGED, (r, st, ns)
    # both FP64 endings describe the same steady state: the switch restored the mass that
    # FP32 rounding had moved
    M1, M2 = s.moments(0), s.moments(2)
    for k in ("n", "T"):
        assert np.max(np.abs(M1[k] - M2[k]) / M2[k]) < 1e-7, k
    for k in ("ux", "qx"):
        assert np.max(np.abs(M1[k] - M2[k])) < 1e-7, k
