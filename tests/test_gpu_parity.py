"""GPU path (through the C ABI) vs the FP64 oracle, element by element on the moments.

FP64 tolerance 1e-12 relative on n, T (absolute on u, scaled), FP32-storage tolerance 1e-5.
Batches mix velocity-space forms, grids and ragged node counts so that tiles, velocity
chunks and the wall closure are all exercised."""
import numpy as np
import pytest

from gpu_common import compare, lib, oracle_for

pytestmark = pytest.mark.gpu

HETERO = [
    dict(nx=50, qx_half=4, qy=4, qz=4, kn=0.1, eta0=0.1, T_left=0.95, T_right=1.05),                  # Fourier, unreduced
    dict(nx=45, qx_half=6, qy=6, qz=0, kn=0.1, eta0=0.2, U_left=-0.42, U_right=0.42, grid="tanh"),     # Couette, reduced 2D
    dict(nx=40, qx_half=4, qy=4, qz=4, kn=0.05, eta0=0.1, accel_y=0.05, j1_shear=True),                # Poiseuille, unreduced
    dict(nx=70, qx_half=5, qy=0, qz=0, kn=0.5, eta0=0.05, T_left=0.9, T_right=1.1),                    # Fourier, reduced 1D
    dict(nx=33, qx_half=8, qy=4, qz=3, kn=0.2, eta0=0.15, U_left=0.1, U_right=-0.2, T_left=1.02, grid="tanh", stretch=1.2),
]


@pytest.mark.parametrize("steps", [1, 150])
def test_heterogeneous_batch_fp64(steps):
    F = lib()
    ps = [F.Params(**kw) for kw in HETERO]
    s = F.Solver(ps)
    s.step(steps)
    for i, p in enumerate(ps):
        o = oracle_for(p)
        assert abs(s.dt[i] - o.dt) <= 1e-15 * o.dt
        o.step(steps)
        compare(s.moments(i), o.moments(), 1e-12, f"instance {i}")
    r, st, nst = s.status()
    assert (st == F.ACTIVE).all() and (nst == steps).all()


def test_first_step_residual_every_instance():
    """Every instance of a batch is anchored at creation: its first residual is the oracle's."""
    F = lib()
    s = F.Solver([F.Params(**d) for d in HETERO])
    s.step(1)
    r, st, ns = s.status()
    assert np.array_equal(s.residual(), r)
    for i, d in enumerate(HETERO):
        o = oracle_for(F.Params(**d))
        o.step(1)
        assert abs(r[i] / o.last_residual - 1.0) < 1e-8, (i, r[i], o.last_residual)


def test_initial_state_matches_oracle():
    F = lib()
    ps = [F.Params(**kw) for kw in HETERO]
    s = F.Solver(ps)
    for i, p in enumerate(ps):
        compare(s.moments(i), oracle_for(p).moments(), 1e-13, f"instance {i}")


def test_fourier_config_5000_steps():
    """Fourier flow, Nx = 50 uniform, walls 0.95/1.05, eta0 = 0.1, Kn = 0.1, 4 half-range
    per side x 4 x 4 (128 velocities), 5000 RK3 steps at CFL 0.5."""
    F = lib()
    p = F.Params(**HETERO[0])
    s = F.Solver([p])
    o = oracle_for(p)
    s.step(5000)
    o.step(5000)
    compare(s.moments(0), o.moments(), 1e-12, "Fourier 5000 steps")
    r, st, nst = s.status()
    assert nst[0] == 5000
    assert abs(r[0] - o.last_residual) <= 1e-12 + 1e-3 * o.last_residual


def test_fp32_storage_within_1e5():
    F = lib()
    ps = [F.Params(**{**kw, "precision": "fp32"}) for kw in HETERO]
    s = F.Solver(ps)
    s.step(300)
    for i, p in enumerate(ps):
        o = oracle_for(p)
        o.step(300)
        Mg, Mo = s.moments(i), o.moments()
        for k in ("n", "T"):
            assert np.max(np.abs(Mg[k] - Mo[k]) / Mo[k]) < 1e-5, (i, k)
        for k in ("ux", "uy"):
            assert np.max(np.abs(Mg[k] - Mo[k])) < 1e-5, (i, k)


def test_mixed_precision_batch():
    """FP64 and FP32-storage instances in one batch each match their own precision's bound."""
    F = lib()
    kw = HETERO[1]
    s = F.Solver([F.Params(**kw), F.Params(**{**kw, "precision": "fp32"})])
    s.step(100)
    o = oracle_for(F.Params(**kw))
    o.step(100)
    compare(s.moments(0), o.moments(), 1e-12, "fp64 member")
    assert np.max(np.abs(s.moments(1)["T"] - o.moments()["T"])) < 1e-5


def test_uniform_equilibrium_stationary_and_mass():
    F = lib()
    rest = F.Params(nx=37, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.2, grid="tanh")
    cou = F.Params(nx=64, qx_half=6, qy=6, qz=0, kn=0.1, eta0=0.2, U_left=-0.42, U_right=0.42, grid="tanh")
    s = F.Solver([rest, cou])
    m0 = [s.moments(i) for i in range(2)]
    o = oracle_for(cou)
    dx = o.dx
    mass0 = np.sum(dx * m0[1]["n"])
    s.step(400)
    M = s.moments(0)
    assert np.max(np.abs(M["n"] - 1.0)) < 1e-13 and np.max(np.abs(M["T"] - 1.0)) < 1e-13
    assert np.max(np.abs(M["uy"])) < 1e-14
    assert abs(np.sum(dx * s.moments(1)["n"]) / mass0 - 1.0) < 1e-13


def test_checkpoint_restart_is_bitwise():
    F = lib()
    p = F.Params(**HETERO[1])
    a = F.Solver([p])
    a.step(60)
    st = a.get_state(0)
    a.step(60)
    b = F.Solver([p])
    b.set_state(0, st)
    b.step(60)
    Ma, Mb = a.moments(0), b.moments(0)
    for k in Ma:
        assert np.array_equal(Ma[k], Mb[k]), k
    assert b.status()[2][0] == 120
    other = F.Solver([F.Params(**HETERO[0])])
    with pytest.raises(F.FdlbError):
        other.set_state(0, st)


def test_set_profiles_round_trip():
    F = lib()
    p = F.Params(**HETERO[1])
    s = F.Solver([p])
    x = np.linspace(-0.5, 0.5, p.nx)
    n = 1.0 + 0.05 * np.cos(np.pi * x)
    uy = 0.3 * x
    T = 1.0 + 0.02 * x * x
    s.set_profiles(0, n, uy, T)
    M = s.moments(0)
    np.testing.assert_allclose(M["n"], n, rtol=1e-13)
    np.testing.assert_allclose(M["uy"], uy, atol=1e-14)
    np.testing.assert_allclose(M["T"], T, rtol=1e-13)
    np.testing.assert_allclose(M["ux"], 0.0, atol=1e-15)
    o = oracle_for(p)
    o.set_profiles(n, uy, T)
    s.step(50)
    o.step(50)
    compare(s.moments(0), o.moments(), 1e-12, "after set_profiles")


def test_residual_freeze_and_status():
    """With a freeze tolerance an instance stops as soon as its per-step residual falls below
    it; the step count and the residual agree with the oracle's own run."""
    F = lib()
    kw = dict(nx=24, qx_half=4, qy=4, qz=0, kn=0.3, eta0=0.1, U_left=-0.2, U_right=0.2, cfl=0.5)
    p = F.Params(**kw)
    s = F.Solver([p])
    tol = 2e-6
    rc = s.run(tol, 20000, check_every=50)
    assert rc == 0
    r, st, nst = s.status()
    assert st[0] == F.CONVERGED and r[0] < tol
    o = oracle_for(p)
    assert o.run_to_residual(tol, 20000)
    assert nst[0] == o.steps
    compare(s.moments(0), o.moments(), 1e-11, "frozen state")


def test_fault_injection_nonfinite():
    """A NaN written into f through the checkpoint path marks the instance FAILED_NONFINITE;
    the other instance keeps stepping; fdlb_run reports FDLB_ENONFINITE."""
    F = lib()
    p = F.Params(**HETERO[1])
    s = F.Solver([p, F.Params(**HETERO[0])])
    st = bytearray(s.get_state(0))
    arr = np.frombuffer(st, dtype=np.float64, offset=24)
    arr[5] = np.nan
    s.set_state(0, bytes(st))
    s.step(3)
    r, status, steps = s.status()
    assert status[0] == F.FAILED_NONFINITE and status[1] == F.ACTIVE
    assert steps[1] == 3
    with pytest.raises(F.FdlbError) as e:
        s.run(1e-30, 10, check_every=5)
    assert e.value.code == F.FDLB_ENONFINITE
