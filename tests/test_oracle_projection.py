"""Pins of the discrete projections (Sec. III A 2 Eqs. hh_F-hh_gk, App. A Eq. H_gk) and the force kernel."""
import math

import numpy as np
import pytest

from oracle import quadrature as qd


def half_line_moments(u, T, smax, a):
    """int_0^inf p^s (p-u)^a g(p;u,T) dp for s <= smax, by integration by parts:
    I_0 = erfc(-u/sqrt(2T))/2, I_1 = u I_0 + T g(0), I_s = u I_{s-1} + (s-1) T I_{s-2};
    then (p-u)^a expanded binomially.  Written here independently of the oracle."""
    g0 = math.exp(-u * u / (2 * T)) / math.sqrt(2 * math.pi * T)
    I = [0.5 * math.erfc(-u / math.sqrt(2 * T))]
    I.append(u * I[0] + T * g0)
    for s in range(2, smax + a + 1):
        I.append(u * I[s - 1] + (s - 1) * T * I[s - 2])
    return [sum(math.comb(a, j) * (-u) ** (a - j) * I[s + j] for j in range(a + 1)) for s in range(smax + 1)]


def full_line_moments(u, T, smax, a):
    M = [1.0, u]
    for s in range(2, smax + a + 1):
        M.append(u * M[s - 1] + (s - 1) * T * M[s - 2])
    return [sum(math.comb(a, j) * (-u) ** (a - j) * M[s + j] for j in range(a + 1)) for s in range(smax + 1)]


@pytest.mark.parametrize("Q", [2, 4, 6, 8])
@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.05, 0.95), (-0.2, 1.1), (0.4, 0.8)])
def test_half_projection_reproduces_moments(Q, u, T):
    """Truncation at order Q-1 reproduces the half-range moments s = 0..Q-1 (reading of Eq. hh_gk)."""
    p = qd.half_range_rule(Q).nodes
    P = qd.project_half(p, u, T)
    for a in range(4):
        want = half_line_moments(u, T, Q - 1, a)
        for s in range(Q):
            got = float(np.sum(P[a] * p ** s))
            assert abs(got - want[s]) < 2e-14 * max(1.0, abs(want[s])), (a, s, got, want[s])
        # negative half-axis: nodes -p_k carry (-1)^a P(-u)
        Pn = (-1) ** a * qd.project_half(p, -u, T)[a]
        wantn = [None] * Q
        for s in range(Q):
            # int_{-inf}^0 (-p)^s (p-u)^a g dp = (-1)^a int_0^inf q^s (q+u)^a g(q;-u,T) dq
            wantn[s] = (-1) ** a * half_line_moments(-u, T, Q - 1, a)[s]
            got = float(np.sum(Pn * p ** s))
            assert abs(got - wantn[s]) < 2e-14 * max(1.0, abs(wantn[s]))


@pytest.mark.parametrize("Q", [1, 2, 4, 8])
def test_half_projection_at_reference_state_is_weights(Q):
    """At u = 0, T = 1 the projected Maxwellian equals the Gauss weights (f_k = w_k, Eq. hh_fk with f = omega)."""
    r = qd.half_range_rule(Q)
    np.testing.assert_allclose(qd.project_half(r.nodes, 0.0, 1.0)[0], r.weights, rtol=1e-13, atol=1e-17)


@pytest.mark.parametrize("Q", [2, 3, 4, 6])
@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.42, 1.05), (-0.7, 0.9)])
def test_full_projection_reproduces_moments(Q, u, T):
    r = qd.full_range_rule(Q)
    P = qd.project_full(r.nodes, u, T)
    for a in range(4):
        want = full_line_moments(u, T, Q - 1, a)
        for s in range(Q):
            got = float(np.sum(P[a] * r.nodes ** s))
            assert abs(got - want[s]) < 1e-13 * max(1.0, abs(want[s]))


def test_full_projection_matches_paper_series():
    """App. A, Eq. (H_gk): g_k = w_k sum_{l<=N} He_l(p_k) sum_s (T-1)^s u^(l-2s)/(2^s s! (l-2s)!), N = Q-1."""
    for Q in (3, 4, 6):
        r = qd.full_range_rule(Q)
        for u, T in ((0.3, 1.2), (-0.42, 0.97)):
            he = [np.ones(Q), r.nodes.copy()]
            for l in range(1, Q):
                he.append(r.nodes * he[l] - l * he[l - 1])
            g = np.zeros(Q)
            for l in range(Q):
                c = sum((T - 1) ** s * u ** (l - 2 * s) / (2 ** s * math.factorial(s) * math.factorial(l - 2 * s)) for s in range(l // 2 + 1))
                g += he[l] * c
            g *= r.weights
            np.testing.assert_allclose(qd.project_full(r.nodes, u, T)[0], g, rtol=1e-12, atol=1e-16)


def test_half_projection_brute_force_mpmath():
    """Brute force: adaptive high-precision quadrature of l_k(p) (p-u)^a g(p) on [0, inf)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    Q = 4
    r = qd.half_range_rule(Q)
    nodes = [mp.mpf(str(x)) for x in r.nodes_dec]
    for u, T in ((0.1, 0.9), (-0.3, 1.2)):
        P = qd.project_half(r.nodes, u, T)
        for k in range(Q):
            for a in range(4):
                def integrand(p):
                    l = mp.mpf(1)
                    for j in range(Q):
                        if j != k:
                            l *= (p - nodes[j]) / (nodes[k] - nodes[j])
                    return l * (p - u) ** a * mp.exp(-(p - u) ** 2 / (2 * T)) / mp.sqrt(2 * mp.pi * T)
                ref = float(mp.quad(integrand, [0, 1, 3, 6, mp.inf]))
                assert abs(P[a, k] - ref) < 1e-15, (k, a, P[a, k], ref)


@pytest.mark.parametrize("Q", [2, 4, 6])
def test_force_kernel(Q):
    """Eq. (kernel_H): columns sum to 0 (mass), sum_k p_k K_kk' = -1 (int p d_p f = -int f),
    and K applied to the projected Maxwellian gives the projection of d_p g = -(p-u)/T g."""
    K = qd.force_matrix(Q)
    r = qd.full_range_rule(Q)
    np.testing.assert_allclose(K.sum(axis=0), 0.0, atol=1e-14)
    np.testing.assert_allclose(r.nodes @ K, -1.0, atol=1e-13)
    for u, T in ((0.2, 1.1), (-0.5, 0.8)):
        P = qd.project_full(r.nodes, u, T)
        np.testing.assert_allclose(K @ P[0], -P[1] / T, atol=1e-14)


@pytest.mark.parametrize("Q", [20, 29])
@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.05, 0.95), (-0.3, 1.1)])
def test_half_projection_high_orders(Q, u, T):
    """The orders of Table 1 (Sec. IV, up to 29 per side): moment exactness s <= Q - 1, relative
    to the sum of the magnitudes of the terms (the high powers of the nodes are large)."""
    p = qd.half_range_rule(Q).nodes
    P = qd.project_half(p, u, T)
    for a in range(4):
        want = half_line_moments(u, T, Q - 1, a)
        for s in range(Q):
            got = float(np.sum(P[a] * p ** s))
            scale = float(np.sum(np.abs(P[a]) * p ** s))
            assert abs(got - want[s]) <= 1e-12 * max(scale, 1.0), (a, s, got, want[s])


@pytest.mark.parametrize("Q", [20, 29])
def test_half_projection_high_orders_reference_state(Q):
    r = qd.half_range_rule(Q)
    np.testing.assert_allclose(qd.project_half(r.nodes, 0.0, 1.0)[0], r.weights, rtol=1e-11, atol=1e-18)


@pytest.mark.parametrize("Q", [24, 40])
def test_full_projection_high_orders(Q):
    """Full-range orders beyond 16 (App. A): weights at rest, moment exactness s <= Q - 1."""
    r = qd.full_range_rule(Q)
    np.testing.assert_allclose(qd.project_full(r.nodes, 0.0, 1.0)[0], r.weights, rtol=1e-10, atol=1e-20)
    u, T = 0.3, 1.05
    P = qd.project_full(r.nodes, u, T)
    for a in range(4):
        want = full_line_moments(u, T, Q - 1, a)
        for s in range(Q):
            got = float(np.sum(P[a] * r.nodes ** s))
            scale = float(np.sum(np.abs(P[a]) * np.abs(r.nodes) ** s))
            assert abs(got - want[s]) <= 1e-12 * max(scale, 1.0), (a, s)


@pytest.mark.parametrize("Q", [64, 100])
def test_half_projection_orders_64_100(Q):
    """Sec. IV's orders for the mass flow at large Kn: at rest the projection is the rule's
    weights (to round-off of the largest weight; the outermost populations, ~1e-60 of the
    largest, keep only absolute accuracy), and at moving states it reproduces the moments
    s <= 8 -- those that carry n, u, T, q and Pi -- of the closed forms above."""
    r = qd.half_range_rule(Q)
    P0 = qd.project_half(r.nodes, 0.0, 1.0)[0]
    assert np.max(np.abs(P0 - r.weights)) <= 1e-14 * r.weights.max()
    big = r.weights > 1e-12 * r.weights.max()
    np.testing.assert_allclose(P0[big], r.weights[big], rtol=1e-9)
    p = r.nodes
    for u, T in ((0.05, 0.95), (-0.3, 1.1)):
        P = qd.project_half(p, u, T)
        for a in range(4):
            want = half_line_moments(u, T, 8, a)
            for s in range(9):
                got = float(np.sum(P[a] * p ** s))
                assert abs(got - want[s]) <= 1e-13 * max(abs(want[s]), 1e-3), (a, s, got, want[s])


@pytest.mark.parametrize("Q", [100, 200])
def test_full_projection_orders_100_200(Q):
    """App. A's orders up to 200: at rest the projection is the rule's weights (to round-off of
    the largest), and at a moving state it reproduces the moments s <= 8 of the closed forms
    (to round-off of the summed terms' magnitudes)."""
    r = qd.full_range_rule(Q)
    P0 = qd.project_full(r.nodes, 0.0, 1.0)[0]
    assert np.max(np.abs(P0 - r.weights)) <= 1e-14 * r.weights.max()
    u, T = 0.3, 1.05
    P = qd.project_full(r.nodes, u, T)
    for a in range(4):
        want = full_line_moments(u, T, 8, a)
        for s in range(9):
            got = float(np.sum(P[a] * r.nodes ** s))
            scale = float(np.sum(np.abs(P[a]) * np.abs(r.nodes) ** s))
            assert abs(got - want[s]) <= 1e-13 * max(scale, abs(want[s])), (a, s, got, want[s])
