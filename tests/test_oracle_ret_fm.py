"""Pins of the oracle's Fischer-Methfessel density average (Eq. chi_ret; reading R15)."""
import math

import numpy as np
import pytest

from oracle import fdlb as ofd


def grid(N, kind="uniform", A=1.5):
    sf = -1.0 + np.arange(N + 1) * 2.0 / N
    s = -1.0 + (np.arange(N) + 0.5) * 2.0 / N
    if kind == "uniform":
        return 0.5 * sf, 0.5 * s
    return 0.5 * np.tanh(A * sf) / math.tanh(A), 0.5 * np.tanh(A * s) / math.tanh(A)


def test_sphere_diameter_from_kn():
    # Kn = 1/(sqrt(2) pi sigma^2 n0 chi0 D) with b n0 = 4 eta0, b = 2 pi sigma^3 / 3
    for eta0, kn in ((0.1, 0.05), (0.2, 0.01), (0.35, 0.1)):
        sigma = ofd.sphere_diameter(eta0, kn)
        n0 = 4.0 * eta0 / (2.0 * math.pi * sigma ** 3 / 3.0)
        kn_back = 1.0 / (math.sqrt(2.0) * math.pi * sigma ** 2 * n0 * float(ofd.chi_set(eta0)))
        assert abs(kn_back / kn - 1.0) < 1e-13


def test_uniform_density_in_the_bulk_is_reproduced():
    faces, x = grid(200)
    W = ofd.ret_fm_weights(faces, x, 0.05)
    inside = np.abs(x) < 0.5 - 0.05
    assert np.max(np.abs(W.sum(axis=1)[inside] - 1.0)) < 1e-14


def test_uniform_density_near_a_wall_closed_form():
    # window cut by the wall at distance d < sigma: 3/(4 s^3) [s^2 d - d^3/3 + 2 s^3/3]
    faces, x = grid(160, "tanh")
    sigma = 0.04
    W = ofd.ret_fm_weights(faces, x, sigma)
    nbar = W @ np.full(x.size, 1.7)
    for i in range(x.size):
        d = min(0.5 - x[i], x[i] + 0.5)
        frac = 1.0 if d >= sigma else 3.0 / (4.0 * sigma ** 3) * (sigma ** 2 * d - d ** 3 / 3.0 + 2.0 * sigma ** 3 / 3.0)
        assert abs(nbar[i] - 1.7 * frac) < 1e-13, i


def test_linear_density_centre_value():
    # uniform grid, window inside: the odd part of the weight integrates to zero
    faces, x = grid(128)
    W = ofd.ret_fm_weights(faces, x, 0.06)
    n = 1.0 + 0.3 * x
    inside = np.abs(x) < 0.5 - 0.06
    assert np.max(np.abs((W @ n - n)[inside])) < 1e-14


def test_small_sphere_is_the_local_density():
    faces, x = grid(50, "tanh")
    dxmin = np.min(np.diff(faces))
    W = ofd.ret_fm_weights(faces, x, 0.4 * dxmin)
    assert np.max(np.abs(W - np.eye(x.size))) < 1e-15


def test_ball_average_brute_force():
    """The 1D weight is the ball average of Eq. chi_ret for n = n(x): Monte Carlo over the
    ball (seeded) against the weight matrix, for a smooth piecewise-constant profile."""
    faces, x = grid(64)
    sigma = 0.09
    W = ofd.ret_fm_weights(faces, x, sigma)
    n = 1.0 + 0.4 * np.sin(7.0 * x) + 0.2 * x
    rng = np.random.Generator(np.random.PCG64(2308))
    # uniform points in the unit ball
    v = rng.normal(size=(400000, 3))
    v *= (rng.random(400000) ** (1.0 / 3.0) / np.linalg.norm(v, axis=1))[:, None]
    for i in (0, 5, 31, 58, 63):
        xs = x[i] + sigma * v[:, 0]
        j = np.searchsorted(faces, xs) - 1
        vals = np.where((xs > -0.5) & (xs < 0.5), n[np.clip(j, 0, x.size - 1)], 0.0)
        assert abs(vals.mean() - W[i] @ n) < 4e-3, i


def test_ret_fm_closure_uses_the_average():
    o = ofd.Oracle(ofd.Params(nx=64, qx_half=4, qy=0, qz=0, kn=0.05, eta0=0.1, chi_model="ret-fm"))
    M = o.moments()
    C = o.nodal(M)
    nbar = o.Wfm @ M["n"]
    assert np.allclose(C["chi"], ofd.chi_set(0.1 * nbar), rtol=1e-15)
    # the walls lower the average: chi_RET < chi_SET at the wall nodes of a uniform state
    assert C["chi"][0] < ofd.chi_set(0.1 * M["n"][0]) and C["chi"][-1] < ofd.chi_set(0.1 * M["n"][-1])
    o2 = ofd.Oracle(ofd.Params(nx=64, qx_half=4, qy=0, qz=0, kn=0.05, eta0=0.1))
    assert np.allclose(C["chi"][20:44], o2.nodal(M)["chi"][20:44], rtol=1e-14)


def test_paper_geometry_parameters():
    """sigma = D/(R - 1) and Delta x = sigma/100 in the paper's confinement; Kn referred to
    L = R sigma is the closed form of Sec. II A (1/(6 sqrt(2) eta0 chi0 R))."""
    from paper_2308_15407_gb300 import workloads
    for R, eta0 in ((4, 0.1), (10, 0.2), (4, 0.01)):
        d = workloads.paper_geometry(R, eta0)
        sigma = ofd.sphere_diameter(eta0, d["kn"])
        assert abs(sigma * (R - 1) - 1.0) < 1e-13
        assert abs((1.0 / d["nx"]) / sigma - 0.01) < 1e-12
        kn_L = d["kn"] * (R - 1) / R
        assert abs(kn_L - ofd.knudsen(eta0, R)) < 1e-15


def test_paper_geometry_flows():
    """The paper's flows in its geometry: walls at T0 -+ dT (Fourier), -+U_0 (Couette), the
    acceleration given in v^2/sigma converted to channel-width units (Poiseuille); every set
    is accepted by the oracle and keeps Delta x = sigma/cells_per_sigma."""
    from paper_2308_15407_gb300 import workloads
    R, eta0 = 10, 0.01
    f = workloads.paper_geometry(R, eta0, flow="fourier", dT=0.5, cells_per_sigma=10)
    assert (f["T_left"], f["T_right"], f["qy"]) == (0.5, 1.5, 0)
    c = workloads.paper_geometry(R, eta0, flow="couette", U_w=1.0, cells_per_sigma=10, x_quadrature="full")
    assert (c["U_left"], c["U_right"], c["qy"], c["x_quadrature"]) == (-1.0, 1.0, 5, "full")
    p = workloads.paper_geometry(R, eta0, flow="poiseuille", a_y=0.001, cells_per_sigma=10)
    sigma = ofd.sphere_diameter(eta0, p["kn"])
    assert abs(p["accel_y"] - 0.001 / sigma) < 1e-15                  # a [v^2/sigma] = a/sigma [v^2/D]
    for d in (f, c, p):
        assert d["nx"] == 90
        keys = {k: v for k, v in d.items() if k not in ("precision",)}
        ofd.Oracle(ofd.Params(**{**keys, "chi_model": "ret-fm"}))
    with pytest.raises(ValueError):
        workloads.paper_geometry(R, eta0, flow="shear")


def test_knudsen_sweep_parameters():
    """The mass-flow sweep's instances: Kn referred to L = R sigma is the closed form of Sec. II A
    at the chosen eta0 (within the stable eta0 <= 0.2), spaced from the smallest reachable Kn to
    1 for each R, in the paper's geometry with the acceleration converted from v^2/sigma."""
    from paper_2308_15407_gb300 import workloads
    dicts, tags = workloads.knudsen_sweep(R_values=(2, 10), points=5)
    assert len(dicts) == 10
    for d, (R, kn, eta0) in zip(dicts, tags):
        assert 0 < eta0 <= 0.2 + 1e-12 and d["eta0"] == eta0
        assert abs(ofd.knudsen(eta0, R) / kn - 1) < 1e-10
        assert abs(d["kn"] * (R - 1) / R / kn - 1) < 1e-10
        assert d["nx"] >= 60 and d["flow"] == 2 and d["chi_model"] == "ret-fm"
        assert abs(d["accel_y"] - 0.001 * (R - 1)) < 1e-15
    kns = [t[1] for t in tags[:5]]
    assert abs(kns[-1] - 1.0) < 1e-12 and all(a < b for a, b in zip(kns, kns[1:]))
    assert workloads.eta_for_knudsen(1e-4, 2) is None
