"""Pins of the oracle's Gauss rules (Sec. III A 2 and App. A)."""
import math
from decimal import Decimal

import numpy as np
import pytest

from oracle import quadrature as qd


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 6, 8, 12])
def test_half_range_exact_moments(Q):
    """Sec. III A 2: the rule is exact for polynomials of degree < 2Q."""
    r = qd.half_range_rule(Q)
    for s in range(2 * Q):
        got = sum(w * x ** s for w, x in zip(r.weights_dec, r.nodes_dec))
        want = qd.half_range_moment(s)
        assert abs(got - want) <= Decimal(10) ** -60 * abs(want)
    # degree 2Q is NOT integrated exactly (checks the rule is not of higher order by accident)
    got = sum(w * x ** (2 * Q) for w, x in zip(r.weights_dec, r.nodes_dec))
    assert abs(got - qd.half_range_moment(2 * Q)) > Decimal(10) ** -30


def test_half_range_moments_closed_form():
    """The moment formula against direct numerical integration (numpy trapezoid on a fine grid)."""
    p = np.linspace(0.0, 40.0, 400001)
    w = np.exp(-p * p / 2) / math.sqrt(2 * math.pi)
    for s in range(9):
        assert abs(np.trapezoid(w * p ** s, p) - float(qd.half_range_moment(s))) < 1e-8 * max(1, float(qd.half_range_moment(s)))


def test_half_range_Q1_closed_form():
    """Q = 1: the node is the mean of omega on [0, inf), sqrt(2/pi), with weight 1/2."""
    r = qd.half_range_rule(1)
    assert abs(r.nodes[0] - math.sqrt(2 / math.pi)) < 1e-15
    assert abs(r.weights[0] - 0.5) < 1e-16


@pytest.mark.parametrize("Q", [1, 2, 4, 6, 8, 12])
def test_half_range_weights_paper_formula(Q):
    """Eq. (hh_wk): w_k = p_k a_Q^2 / (h_{Q+1}(p_k)^2 [p_k + h_Q(0)^2/sqrt(2 pi)]), a_Q = h_{Q+1,Q+1}/h_{Q,Q}."""
    r = qd.half_range_rule(Q)
    aQ = r.ortho[Q + 1][Q + 1] / r.ortho[Q][Q]
    s2pi = (2 * qd._pi()).sqrt()
    for x, w in zip(r.nodes_dec, r.weights_dec):
        wp = x * aQ ** 2 / (r.eval_ortho(Q + 1, x) ** 2 * (x + r.eval_ortho(Q, Decimal(0)) ** 2 / s2pi))
        assert abs(wp - w) <= Decimal(10) ** -50 * w


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 5, 6, 8])
def test_full_range_matches_hermegauss(Q):
    """Library special case: numpy's probabilists' Gauss-Hermite rule (weights / sqrt(2 pi))."""
    r = qd.full_range_rule(Q)
    x, w = np.polynomial.hermite_e.hermegauss(Q)
    np.testing.assert_allclose(r.nodes, x, atol=1e-13)
    np.testing.assert_allclose(r.weights, w / math.sqrt(2 * math.pi), rtol=1e-13)


@pytest.mark.parametrize("Q", [2, 3, 4, 6, 8])
def test_full_range_weights_paper_formula(Q):
    """App. A, Eq. (H_wk): w_k = Q!/He_{Q+1}(p_k)^2."""
    r = qd.full_range_rule(Q)
    for x, w in zip(r.nodes_dec, r.weights_dec):
        he = [Decimal(1), x]
        for l in range(1, Q + 1):
            he.append(x * he[l] - l * he[l - 1])
        assert abs(Decimal(math.factorial(Q)) / he[Q + 1] ** 2 - w) <= Decimal(10) ** -50 * w


@pytest.mark.parametrize("Q", [64, 100])
def test_half_range_high_orders(Q):
    """The orders Sec. IV uses for the mass flow at large Kn (64, and 100 above Kn = 1): exact
    moments below degree 2Q; at degree 2Q the rule misses by exactly the squared norm of the
    monic pi_Q (it integrates p^2Q - pi_Q^2 exactly and pi_Q vanishes at the nodes), which pins
    the nodes as the zeros of pi_Q (decimal); the weights of Eq. (hh_wk); and the float64
    rule exact to round-off relative to the terms' magnitudes; the working precision grows with
    the order (the moment route loses digits), which a 200-digit build would not reach."""
    r = qd.half_range_rule(Q)
    assert r.prec > 200
    for s in range(0, 2 * Q, 3):
        got = sum(w * x ** s for w, x in zip(r.weights_dec, r.nodes_dec))
        assert abs(got - qd.half_range_moment(s)) <= Decimal(10) ** -60 * qd.half_range_moment(s)
    got = sum(w * x ** (2 * Q) for w, x in zip(r.weights_dec, r.nodes_dec))
    miss = qd.half_range_moment(2 * Q) - got
    assert abs(miss - r.norms[Q]) <= Decimal(10) ** -40 * r.norms[Q]
    aQ = r.ortho[Q + 1][Q + 1] / r.ortho[Q][Q]
    s2pi = (2 * qd._pi()).sqrt()
    for x, w in list(zip(r.nodes_dec, r.weights_dec))[::7]:
        wp = x * aQ ** 2 / (r.eval_ortho(Q + 1, x) ** 2 * (x + r.eval_ortho(Q, Decimal(0)) ** 2 / s2pi))
        assert abs(wp - w) <= Decimal(10) ** -40 * w
    x, w = r.nodes, r.weights
    assert np.all(np.diff(x) > 0) and np.all(w > 0)
    for s in range(2 * Q):
        got = np.sum(w * x ** s)
        assert abs(got - float(qd.half_range_moment(s))) <= 1e-13 * np.sum(w * x ** s)
