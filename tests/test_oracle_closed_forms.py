"""Pins of the Sec. II closed forms, the FD stencils, WENO-5 and the golden constants."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import fdlb as ofd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        vals = []
        for tok in parts[1:]:
            try:
                vals.append(Fraction(tok))
            except ValueError:
                break
        out[parts[0]] = vals
    return out


def test_chi_values():
    assert float(ofd.chi_set(0.0)) == 1.0
    assert abs(float(ofd.chi_set(0.1)) - 1.9 / 1.458) < 1e-15       # (2-0.1)/(2*0.9^3)


def test_chi_from_eos():
    """Eq. (chi) = (P^hs/(n k_B T) - 1)/(n b) with Eq. (eos) and n b = 4 eta."""
    eta = np.linspace(0.0, 0.49, 50)
    lhs = ofd.chi_set(eta)
    rhs = np.where(eta > 0, (ofd.eos_ratio(eta) - 1.0) / np.where(eta > 0, 4 * eta, 1.0), 1.0)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_prandtl_from_mu_and_lambda():
    """Eq. (prandtl) equals c_P mu/lambda with mu, lambda of Eqs. (viscosity) and the lambda line,
    lambda0/mu0 = (75/64)/(5/16) = 15/4, c_P = 5/2."""
    for eta in (0.0, 0.05, 0.2, 0.4):
        chi = float(ofd.chi_set(eta))
        br = 4 * eta
        mu = 1 / chi + 0.8 * br + 4 / 25 * (1 + 12 / math.pi) * br ** 2 * chi
        lam = 15 / 4 * (1 / chi + 1.2 * br + 9 / 25 * (1 + 32 / (9 * math.pi)) * br ** 2 * chi)
        assert abs(float(ofd.prandtl(br * chi)) - 2.5 * mu / lam) < 1e-14
    g = golden()
    assert float(ofd.prandtl(0.0)) == float(g["prandtl_dilute"][0])


def test_knudsen_and_mu0():
    """Kn = 1/(6 sqrt2 eta0 chi0 R) (Sec. II A); mu0 = 5/(16 sigma^2) sqrt(T/pi) with
    sigma^2 = 1/(sqrt2 pi n0 chi0 Kn L), n0 = L = 1 (reading R1)."""
    assert abs(ofd.knudsen(0.1, 10.0) - 1 / (6 * math.sqrt(2) * 0.1 * (1.9 / 1.458) * 10)) < 1e-15
    assert abs(ofd.knudsen(0.1, 10.0) - 0.0904352357) < 1e-9
    for kn, eta0, T in ((0.1, 0.1, 1.0), (0.05, 0.3, 1.2)):
        chi0 = float(ofd.chi_set(eta0))
        sigma2 = 1 / (math.sqrt(2) * math.pi * chi0 * kn)
        assert abs(float(ofd.mu0(T, kn, eta0)) - 5 / (16 * sigma2) * math.sqrt(T / math.pi)) < 1e-15
    # the same Kn from sigma and eta0 = b n0/4 = (2 pi sigma^3/3)/4 in the R form: L = R sigma
    eta0 = 0.2
    R = 4.0
    kn = ofd.knudsen(eta0, R)
    chi0 = float(ofd.chi_set(eta0))
    sigma = (6 * eta0 / math.pi) ** (1 / 3)          # n0 = 1: eta0 = pi sigma^3/6
    L = R * sigma
    assert abs(kn - 1 / (math.sqrt(2) * math.pi * sigma ** 2 * chi0 * L)) < 1e-13


def test_viscosity_dilute_limit():
    """eta -> 0: chi = 1, b rho = 0, mu = mu0."""
    assert abs(float(ofd.viscosity(1.0, 1.3, 0.2, 0.0)) - float(ofd.mu0(1.3, 0.2, 0.0))) < 1e-16


def test_fd6_central_matches_paper():
    g = golden()["fd6_central"]
    w = ofd.fd_weights(list(range(-3, 4)), 0)
    assert w == g


def test_fd_one_sided_textbook():
    """7-point one-sided first derivative at the end node: (-49/20, 6, -15/2, 20/3, -15/4, 6/5, -1/6)."""
    w = ofd.fd_weights(list(range(7)), 0)
    assert w == [Fraction(-49, 20), 6, Fraction(-15, 2), Fraction(20, 3), Fraction(-15, 4), Fraction(6, 5), Fraction(-1, 6)]


@pytest.mark.parametrize("N", [8, 12, 30])
def test_gradient_matrix_exact_for_degree_6(N):
    D = ofd.gradient_matrix(N)
    i = np.arange(N, dtype=float)
    for k in range(7):
        want = k * i ** (k - 1) if k else np.zeros(N)
        np.testing.assert_allclose(D @ i ** k, want, rtol=1e-10, atol=1e-8)
    # degree 7 is not exact at the central nodes (6th order, not higher)
    assert np.abs(D @ i ** 7 - 7 * i ** 6)[3:N - 3].max() > 1.0


def test_weno_constants_match_paper():
    g = golden()
    assert [float(x) for x in g["weno_ideal"]] == list(ofd.DELTA)
    eye = np.eye(5)
    F = ofd.weno5_candidates(*[eye[:, j] for j in range(5)])
    for q, name in enumerate(("weno_F1", "weno_F2", "weno_F3")):
        np.testing.assert_allclose(F[q], [float(x) for x in g[name]], atol=1e-15)


def test_weno_uniform_and_quadratic():
    """Uniform data -> face value equals the data; quadratic data -> all candidates coincide."""
    v = [np.full(7, 0.37)] * 5
    face = ofd.weno5_face(*v)
    assert abs(face[0] - 0.37) < 1e-16 and np.all(np.diff(face) == 0.0)   # zero flux difference exactly
    xs = np.arange(-2, 3, dtype=float)
    quad = 0.3 + 0.2 * xs - 0.05 * xs ** 2
    F = ofd.weno5_candidates(*[np.array([q]) for q in quad])
    assert abs(F[0][0] - F[1][0]) < 1e-15 and abs(F[1][0] - F[2][0]) < 1e-15


def test_weno_limiting_cases():
    """A vanishing indicator takes the whole weight (the limit of delta_q/phi_q^2)."""
    one = lambda x: np.array([float(x)])
    # phi_2 = 0 only: central stencil flat
    assert abs(ofd.weno5_face(one(3), one(1), one(1), one(1), one(5))[0] - 1.0) < 1e-15
    # phi_1 = 0 only: left stencil flat, right one not
    F1 = ofd.weno5_face(one(2), one(2), one(2), one(4), one(9))
    assert abs(F1[0] - 2.0) < 1e-15
    # phi_1 = phi_2 = 0 is impossible without phi_3 = 0 ... check phi_3 = 0 only
    F3 = ofd.weno5_face(one(9), one(4), one(2), one(2), one(2))
    assert abs(F3[0] - 2.0) < 1e-15


def test_weno_fifth_order_convergence():
    """Smooth monotone data (f' != 0, where the epsilon-free weights stay within O(h^2) of
    the ideal ones): the flux difference converges at 5th order to f'.  Near critical points
    epsilon-free Jiang-Shu weights lose order, so the profile has none."""
    errs = []
    for N in (40, 80, 160):
        h = 1.0 / N
        x = np.arange(-3, N + 4) * h
        f = np.exp(x) + 0.5 * x
        v = lambda k: f[k:k + N + 2]                            # f_{i+k-2} for faces i+1/2, i = -1..N
        face = ofd.weno5_face(v(0), v(1), v(2), v(3), v(4))    # faces i+1/2, i = -1 .. N
        deriv = (face[1:] - face[:-1]) / h                      # nodes 0..N
        exact = np.exp(x[3:3 + len(deriv)]) + 0.5
        errs.append(np.abs(deriv - exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 4.7, rates
