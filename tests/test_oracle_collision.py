"""Pins of the discrete Shakhov target and J1 (Sec. II A, Eqs. j0, j1) through their moments.

The identities below follow from Gaussian moments of the 3D polynomials, e.g.
E[xi_x^2 |xi|^2] = 5T^2, E[|xi|^4] = 15T^2, E[xi_x^2 |xi|^4] = 35 T^3.  They hold for the
discrete values exactly (to round-off) once Q_x^h >= 4, Q_y >= 4, Q_z >= 3, because the
projection reproduces every moment of degree <= 3 per axis."""
import numpy as np
import pytest

from oracle import fdlb as ofd

STATES = dict(n=np.array([1.0, 0.8, 1.3]), ux=np.array([0.0, 0.03, -0.05]),
              uy=np.array([0.0, 0.42, -0.2]), T=np.array([1.0, 0.9, 1.15]),
              qx=np.array([0.0, 0.02, -0.03]), qy=np.array([0.0, -0.01, 0.04]))
GRADS = dict(G=np.array([0.3, -0.7, 1.1]), B=np.array([0.2, 0.5, -0.4]),
             U=np.array([0.1, -0.3, 0.25]), V=np.array([-0.6, 0.4, 0.9]))


def make(qy, qz, shear=False):
    return ofd.Oracle(ofd.Params(nx=8, qx_half=4, qy=qy, qz=qz, kn=0.1, eta0=0.1, j1_shear=shear))


def discrete_moments(o, h, M):
    px = o.px[:, None, None]
    py = o.py[None, :, None]
    mt = o.mt[None, :, None]
    et = o.et[None, :, None]
    xx = px - M["ux"]
    xy = py - M["uy"]
    E = mt * 0.5 * (xx ** 2 + xy ** 2) + et
    S = lambda w: np.sum(w * h, axis=(0, 1))
    return dict(mass=S(mt), mx=S(mt * xx), my=S(mt * xy), E=S(E), qx=S(xx * E), qy=S(xy * E),
                Pxx=S(mt * xx * xx), Pxy=S(mt * xx * xy))


FORMS = [(4, 4), (4, 0), (6, 3)]


@pytest.mark.parametrize("qy,qz", FORMS)
@pytest.mark.parametrize("shear", [False, True])
def test_j1_moments(qy, qz, shear):
    o = make(qy, qz, shear)
    M = dict(STATES)
    brc = np.array([0.5, 0.9, 1.7])
    tau = np.array([0.1, 0.2, 0.05])
    C = dict(Pr=np.ones(3), tau=tau, brc=brc, **GRADS)       # Pr = 1 switches the Shakhov term off
    J1 = (o.target(M, C) - o.equilibrium(M["n"], M["ux"], M["uy"], M["T"])) / tau
    m = discrete_moments(o, J1, M)
    n, T = M["n"], M["T"]
    G, B, U, V = GRADS["G"], GRADS["B"], GRADS["U"], GRADS["V"]
    tol = 1e-13
    np.testing.assert_allclose(m["mass"], 0.0, atol=tol)
    np.testing.assert_allclose(m["mx"], -brc * n * T * G, rtol=1e-12, atol=tol)      # -d_x(b rho^2 chi T)
    np.testing.assert_allclose(m["my"], 0.0, atol=tol)
    np.testing.assert_allclose(m["E"], -brc * n * T * U, rtol=1e-12, atol=tol)       # collisional work
    np.testing.assert_allclose(m["qx"], -brc * n * T ** 2 * (2.5 * G + 1.5 * B), rtol=1e-12, atol=tol)
    np.testing.assert_allclose(m["qy"], 0.0, atol=tol)
    np.testing.assert_allclose(m["Pxx"], -1.2 * brc * n * T * U, rtol=1e-12, atol=tol)
    np.testing.assert_allclose(m["Pxy"], -0.4 * brc * n * T * V * (1.0 if shear else 0.0), rtol=1e-12, atol=tol)


@pytest.mark.parametrize("qy,qz", FORMS)
def test_j1_vanishes(qy, qz):
    """J1 = 0 for zero gradients and for b rho chi = 0 (eta0 -> 0)."""
    o = make(qy, qz, True)
    M = dict(STATES)
    Mfs = dict(M, qx=np.zeros(3), qy=np.zeros(3))
    eq = o.equilibrium(M["n"], M["ux"], M["uy"], M["T"])
    zero = {k: np.zeros(3) for k in GRADS}
    C = dict(Pr=np.ones(3), tau=np.full(3, 0.1), brc=np.full(3, 0.8), **zero)
    np.testing.assert_allclose(o.target(Mfs, C), eq, atol=1e-16)
    C = dict(Pr=np.ones(3), tau=np.full(3, 0.1), brc=np.zeros(3), **GRADS)
    np.testing.assert_allclose(o.target(Mfs, C), eq, atol=1e-16)


@pytest.mark.parametrize("qy,qz", FORMS)
def test_shakhov_moments(qy, qz):
    """Collision invariants of f^S equal those of f, its heat flux is (1 - Pr) q, its stress is n T I."""
    o = make(qy, qz)
    M = dict(STATES)
    Pr = np.array([2 / 3, 0.7, 0.55])
    C = dict(Pr=Pr, tau=np.full(3, 0.1), brc=np.zeros(3), **{k: np.zeros(3) for k in GRADS})
    fS = o.target(M, C)
    m = discrete_moments(o, fS, M)
    n, T = M["n"], M["T"]
    np.testing.assert_allclose(m["mass"], n, rtol=1e-13)
    np.testing.assert_allclose(m["mx"], 0.0, atol=1e-14)
    np.testing.assert_allclose(m["my"], 0.0, atol=1e-14)
    np.testing.assert_allclose(m["E"], 1.5 * n * T, rtol=1e-13)
    np.testing.assert_allclose(m["qx"], (1 - Pr) * M["qx"], atol=1e-14)
    np.testing.assert_allclose(m["qy"], (1 - Pr) * M["qy"], atol=1e-14)
    np.testing.assert_allclose(m["Pxx"], n * T, rtol=1e-13)
    np.testing.assert_allclose(m["Pxy"], 0.0, atol=1e-14)
    # and the oracle's own moment routine reads the equilibrium back exactly
    Mr = o.moments(o.equilibrium(M["n"], M["ux"], M["uy"], M["T"]))
    for k in ("n", "ux", "uy", "T"):
        np.testing.assert_allclose(Mr[k], M[k], rtol=1e-13, atol=1e-14)


def test_reduced_forms_are_transverse_moments_of_unreduced():
    """phi = sum_kz f, theta = sum_kz p_z^2 f (Sec. II B 2), and phi_1D, theta_1D over (p_y, p_z)
    (Sec. II B 1): the reduced targets equal the transverse moments of the unreduced one."""
    M = dict(STATES)
    C = dict(Pr=np.array([0.6, 0.66, 0.7]), tau=np.full(3, 0.07), brc=np.array([0.4, 0.8, 1.2]), **GRADS)
    u = make(4, 4, True)
    r2 = make(4, 0, True)
    tu = u.target(M, C).reshape(8, 4, 4, 3)           # [kx, ky, kz, i]
    t2 = r2.target(M, C).reshape(8, 4, 2, 3)          # [kx, ky, slot, i]
    z = u.zrule.nodes
    np.testing.assert_allclose(tu.sum(axis=2), t2[:, :, 0], atol=1e-15)
    np.testing.assert_allclose(np.einsum("xyzi,z->xyi", tu, z * z), t2[:, :, 1], atol=1e-15)
    # 1D: only valid without y dynamics
    M1 = dict(M, uy=np.zeros(3), qy=np.zeros(3))
    C1 = dict(C, V=np.zeros(3))
    u1 = ofd.Oracle(ofd.Params(nx=8, qx_half=4, qy=4, qz=4, kn=0.1, eta0=0.1))
    r1 = ofd.Oracle(ofd.Params(nx=8, qx_half=4, qy=0, qz=0, kn=0.1, eta0=0.1))
    tu = u1.target(M1, C1).reshape(8, 4, 4, 3)
    t1 = r1.target(M1, C1)
    y = u1.yrule.nodes
    np.testing.assert_allclose(tu.sum(axis=(1, 2)), t1[:, 0], atol=1e-15)
    perp = (y[:, None] ** 2 + z[None, :] ** 2)
    np.testing.assert_allclose(np.einsum("xyzi,yz->xi", tu, perp), t1[:, 1], atol=1e-15)
