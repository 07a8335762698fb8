"""Oracle pins for the full-range x quadrature (App. A; reading R16): the rule of even order
2 Q_x^h against numpy's Gauss-HermiteE rule, exactness of the discrete equilibrium up to
order 2 Q_x^h - 1 from Gaussian closed forms, free-molecular Fourier and Couette flows against
the closed forms of the discrete problem (built here from numpy's nodes and monomial
Lagrange coefficients, not from the oracle's projection routine), and the invariants
(stationarity, mass, mirror symmetry)."""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He
from numpy.polynomial import polynomial as Pn

from oracle import fdlb as ofd


def gauss_raw(s, T):
    """E[z^s] T^(s/2) for z standard normal: (s-1)!! T^(s/2), 0 for odd s."""
    if s % 2:
        return 0.0
    return float(np.prod(np.arange(s - 1, 0, -2))) * T ** (s // 2)


def shifted_moment(a, s, u, T):
    """E[(p - u)^a p^s] for p ~ N(u, T), by the binomial expansion of p = u + (p - u)."""
    return sum(math.comb(s, j) * u ** (s - j) * gauss_raw(a + j, T) for j in range(s + 1))


def numpy_rule(order):
    x, w = He.hermegauss(order)
    return x, w / math.sqrt(2 * math.pi)


def layout(order):
    """Nodes and weights in the solver's order: +p_1..+p_Q, then -p_1..-p_Q."""
    x, w = numpy_rule(order)
    pos = x > 0
    p, wp = x[pos], w[pos]
    o = np.argsort(p)
    return np.concatenate([p[o], -p[o]]), np.concatenate([wp[o], wp[o]])


def wall_values(order, T):
    """int l_k(p) g(p; 0, T) dp on the full-range nodes (solver order), from the monomial
    coefficients of the Lagrange polynomials and the Gaussian moments."""
    x, _ = layout(order)
    out = np.empty(order)
    for k in range(order):
        roots = np.delete(x, k)
        c = Pn.polyfromroots(roots) / np.prod(x[k] - roots)
        out[k] = sum(c[s] * gauss_raw(s, T) for s in range(len(c)))
    return out


@pytest.mark.parametrize("Q", [2, 4, 8])
def test_nodes_and_rest_values(Q):
    o = ofd.Oracle(ofd.Params(nx=8, qx_half=Q, qy=0, qz=0, kn=0.1, eta0=0.1, x_quadrature="full"))
    x, w = layout(2 * Q)
    np.testing.assert_allclose(o.px, x, rtol=1e-13)
    P = o.x_projection(np.zeros(1), np.ones(1))[:, :, 0]
    # at u = 0, T = 1 the Gauss rule integrates l_k(p) p^a exactly (degree 2Q - 1 + a < 4Q):
    # P[a][k] = w_k p_k^a
    for a in range(4):
        np.testing.assert_allclose(P[a], w * x ** a, rtol=1e-11, atol=1e-15)
    # the ordering matters for the dt rule (largest node) and the wall split (first Q positive)
    assert np.all(o.px[:Q] > 0) and np.all(o.px[Q:] < 0)


@pytest.mark.parametrize("Q", [3, 4, 8])
def test_projection_reproduces_moments_to_order_2Q_minus_1(Q):
    o = ofd.Oracle(ofd.Params(nx=8, qx_half=Q, qy=0, qz=0, kn=0.1, eta0=0.1, x_quadrature="full"))
    u = np.array([0.0, 0.31, -0.55, 0.12])
    T = np.array([1.0, 0.8, 1.3, 1.05])
    P = o.x_projection(u, T)                                             # [a, k, i]
    for i in range(len(u)):
        for a in range(4):
            for s in range(2 * Q):
                terms = P[a, :, i] * o.px ** s
                got = float(np.sum(terms))
                ref = shifted_moment(a, s, u[i], T[i])
                # rounding of the sum scales with its largest terms (p_k^s reaches 1e10)
                assert abs(got - ref) <= 1e-12 * max(1.0, float(np.sum(np.abs(terms)))), (i, a, s, got, ref)
    # order 2Q is not reproduced at u != 0 (the expansion is truncated at 2Q - 1)
    got = float(np.sum(P[0, :, 1] * o.px ** (2 * Q)))
    assert abs(got - shifted_moment(0, 2 * Q, u[1], T[1])) > 1e-6


def test_free_molecular_fourier_discrete_closed_form():
    """eta0 = 0, Kn -> inf: every x-velocity carries its wall's discrete Maxwellian,
    phi_k = n_w P_k(T_w), theta_k = 2 T_w phi_k; n_L, n_R from zero net mass flux and the
    total mass.  The full-range rule does not integrate the half-range Maxwellians exactly, so
    the flux misses the continuous closed form by several per cent at 8 velocities."""
    Q, TL, TR = 4, 0.9, 1.1
    o = ofd.Oracle(ofd.Params(nx=8, qx_half=Q, qy=0, qz=0, kn=1e12, eta0=0.0, T_left=TL, T_right=TR, cfl=1.0,
                              x_quadrature="full"))
    o.step(2400)
    M = o.moments()
    x, _ = layout(2 * Q)
    PL, PR = wall_values(2 * Q, TL), wall_values(2 * Q, TR)
    pos = x > 0
    A = np.array([[np.sum((x * PL)[pos]), np.sum((x * PR)[~pos])],
                  [np.sum(PL[pos]), np.sum(PR[~pos])]])
    nL, nR = np.linalg.solve(A, [0.0, 1.0])
    phi = np.where(pos, nL * PL, nR * PR)
    Tw = np.where(pos, TL, TR)
    qex = float(np.sum(x * (0.5 * x * x * phi + Tw * phi)))
    assert np.abs(M["qx"] / qex - 1).max() < 1e-10
    assert np.abs(M["n"] - 1).max() < 1e-10
    qcont = 4 / math.sqrt(2 * math.pi) * math.sqrt(TL * TR) / (math.sqrt(TL) + math.sqrt(TR)) * (TL - TR)
    assert 0.03 < qex / qcont - 1 < 0.10


def test_free_molecular_couette_discrete_closed_form():
    """eta0 = 0, Kn -> inf, walls at T = 1: n_w = 1 and Pi_xy = -(U_R - U_L) sum_{p_k > 0} w_k p_k
    (the full-range weights stand in for the half-range flux 1/sqrt(2 pi))."""
    Q, UL, UR = 4, -0.3, 0.42
    o = ofd.Oracle(ofd.Params(nx=8, qx_half=Q, qy=4, qz=0, kn=1e12, eta0=0.0, U_left=UL, U_right=UR, cfl=1.0,
                              x_quadrature="full"))
    o.step(1200)
    M = o.moments()
    x, w = layout(2 * Q)
    pex = -(UR - UL) * float(np.sum((w * x)[:Q]))
    assert np.abs(M["Pxy"] / pex - 1).max() < 1e-10
    np.testing.assert_allclose(M["uy"], 0.5 * (UL + UR), atol=1e-10)


@pytest.mark.parametrize("qy,qz", [(4, 4), (4, 0), (0, 0)])
def test_rest_state_is_stationary(qy, qz):
    o = ofd.Oracle(ofd.Params(nx=12, qx_half=4, qy=qy, qz=qz, kn=0.1, eta0=0.2, grid="tanh", x_quadrature="full"))
    f0 = o.f.copy()
    o.step(30)
    assert np.abs(o.f - f0).max() <= 1e-13 * np.abs(f0).max()


def test_mass_and_mirror_symmetry():
    o = ofd.Oracle(ofd.Params(nx=16, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.2, U_left=-0.42, U_right=0.42,
                              grid="tanh", x_quadrature="full"))
    m0 = o.mass()
    o.step(100)
    assert abs(o.mass() / m0 - 1) < 5e-14
    M = o.moments()
    np.testing.assert_allclose(M["uy"], -M["uy"][::-1], atol=1e-13)
    np.testing.assert_allclose(M["n"], M["n"][::-1], rtol=1e-13)
    np.testing.assert_allclose(M["T"], M["T"][::-1], rtol=1e-13)
    a = ofd.Oracle(ofd.Params(nx=16, qx_half=3, qy=0, qz=0, kn=0.2, eta0=0.1, T_left=0.9, T_right=1.1,
                              x_quadrature="full"))
    b = ofd.Oracle(ofd.Params(nx=16, qx_half=3, qy=0, qz=0, kn=0.2, eta0=0.1, T_left=1.1, T_right=0.9,
                              x_quadrature="full"))
    a.step(80)
    b.step(80)
    Ma, Mb = a.moments(), b.moments()
    np.testing.assert_allclose(Ma["T"], Mb["T"][::-1], rtol=1e-13)
    np.testing.assert_allclose(Ma["qx"], -Mb["qx"][::-1], atol=1e-13)


def test_unknown_quadrature_rejected():
    with pytest.raises(ValueError):
        ofd.Oracle(ofd.Params(nx=8, qx_half=4, qy=0, qz=0, kn=0.1, eta0=0.1, x_quadrature="gauss"))
