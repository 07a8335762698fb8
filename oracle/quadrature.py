"""Gauss quadratures and discrete projections for the FDLB velocity space (oracle).

Test infrastructure only (see ``oracle/__init__``).

Sources in the paper:
  * Sec. III A 2 (half-range Gauss-Hermite): weight omega(p) = exp(-p^2/2)/sqrt(2 pi)
    on [0, inf) (the printed exponent has a lost minus sign; the full-range weight
    of App. A, Eq. (A4), fixes it), nodes = positive roots of the orthonormal
    half-range Hermite polynomial h_Q, exactness for degree < 2Q, closed-form
    weights Eq. (hh_wk).
  * App. A (full-range Gauss-Hermite): nodes = roots of He_Q, weights
    Q!/He_{Q+1}(p_k)^2, exact for degree < 2Q.
  * Sec. III A 2, Eqs. (hh_F)-(hh_gk) and App. A, Eq. (H_gk): the discrete
    equilibrium is the expansion of f^eq in the axis' orthogonal polynomials
    truncated at order Q-1.  Truncation at Q-1 is the same as requiring that the
    Q discrete values reproduce the first Q moments (s = 0..Q-1) of the function on
    that (half-)axis, i.e. value_k = integral of l_k(p) h(p) dp with l_k the
    Lagrange basis polynomial of node k (Christoffel-Darboux).  That integral is
    what ``project_half`` / ``project_full`` evaluate.

All rules are built from exact moments in decimal arithmetic of at least 200
digits (Stieltjes procedure on the moment functional, Newton-polished roots,
Christoffel weights) and only then rounded to float64.  The moment route loses
digits with the order (the Hankel matrix of the moments is ill-conditioned), so
orders above 46 work with 60 + 3 Q digits.
"""
from __future__ import annotations

import functools
import math
from decimal import Decimal, getcontext, localcontext

import numpy as np

_PREC = 200
_prec_now = [_PREC]          # working precision of the rule being built


def _rule_prec(Q: int) -> int:
    return max(_PREC, 60 + 3 * Q)


def _ctx():
    getcontext().prec = _prec_now[0]


def _pi() -> Decimal:
    """pi to the working precision by Machin's formula 4 atan(1/5) - atan(1/239)."""
    _ctx()

    def atan_inv(n: int) -> Decimal:
        x = Decimal(1) / n
        x2 = x * x
        term, total, k = x, x, 1
        eps = Decimal(10) ** (-(_prec_now[0] + 5))
        while abs(term) > eps:
            term *= -x2
            total += term / (2 * k + 1)
            k += 1
        return total

    return 4 * (4 * atan_inv(5) - atan_inv(239))


def half_range_moment(s: int) -> Decimal:
    """int_0^inf p^s exp(-p^2/2)/sqrt(2 pi) dp.

    Even s = 2m: (2m-1)!!/2.  Odd s = 2m+1: 2^m m!/sqrt(2 pi)."""
    _ctx()
    if s % 2 == 0:
        r = Decimal(1)
        for j in range(1, s, 2):
            r *= j
        return r / 2
    m = (s - 1) // 2
    return Decimal(2) ** m * math.factorial(m) / (2 * _pi()).sqrt()


def full_range_moment(s: int) -> Decimal:
    """int_R p^s exp(-p^2/2)/sqrt(2 pi) dp = (s-1)!! for even s, 0 for odd s."""
    if s % 2:
        return Decimal(0)
    r = Decimal(1)
    for j in range(1, s, 2):
        r *= j
    return r


class GaussRule:
    """Gauss rule of order Q for a positive weight given by its moments.

    Holds the monic recurrence pi_{l+1} = (p - alpha_l) pi_l - beta_l pi_{l-1},
    the orthonormal polynomials' monomial coefficients (decimal), the nodes and
    Christoffel weights (decimal and float64)."""

    def __init__(self, Q: int, moment):
        prev = _prec_now[0]
        _prec_now[0] = _rule_prec(Q)
        try:
            self._build(Q, moment)
        finally:
            _prec_now[0] = prev
            _ctx()

    def _build(self, Q: int, moment):
        _ctx()
        prec = _prec_now[0]
        self.prec = prec
        self.Q = Q
        mom = [moment(s) for s in range(2 * Q + 4)]

        def ip(a, b):
            return sum(a[i] * b[j] * mom[i + j] for i in range(len(a)) for j in range(len(b)) if a[i] and b[j])

        # Stieltjes procedure on the moment functional, monic polynomials.
        monic = [[Decimal(1)]]
        norms = [ip(monic[0], monic[0])]
        alpha, beta = [], [Decimal(0)]
        for l in range(Q + 1):
            pl = monic[l]
            xpl = [Decimal(0)] + pl
            al = ip(xpl, pl) / norms[l]
            alpha.append(al)
            nxt = [Decimal(0)] * (l + 2)
            for i, c in enumerate(xpl):
                nxt[i] += c
            for i, c in enumerate(pl):
                nxt[i] -= al * c
            if l > 0:
                bl = norms[l] / norms[l - 1]
                beta.append(bl)
                for i, c in enumerate(monic[l - 1]):
                    nxt[i] -= bl * c
            monic.append(nxt)
            norms.append(ip(nxt, nxt))
        self.alpha = alpha          # alpha_0 .. alpha_{Q+1}
        self.beta = beta            # beta_0 = 0, beta_1 .. beta_{Q+1}
        self.monic = monic          # pi_0 .. pi_{Q+2}
        self.norms = norms
        # orthonormal polynomials h_l = pi_l / sqrt(<pi_l, pi_l>), coefficient lists
        self.ortho = [[c / norms[l].sqrt() for c in monic[l]] for l in range(Q + 2)]

        # Nodes: eigenvalues of the float64 Jacobi matrix as starting points,
        # then Newton on pi_Q in decimal arithmetic.
        J = np.diag([float(a) for a in alpha[:Q]])
        off = [float(b.sqrt()) for b in beta[1:Q]]
        J = J + np.diag(off, 1) + np.diag(off, -1)
        guesses = np.sort(np.linalg.eigvalsh(J)) if Q > 0 else []
        nodes = []
        for g in guesses:
            x = Decimal(repr(float(g)))
            for _ in range(100):
                f, df = self._eval_monic_with_derivative(Q, x)
                dx = f / df
                x -= dx
                if abs(dx) < Decimal(10) ** (-(prec - 20)):
                    break
            nodes.append(x)
        self.nodes_dec = nodes
        self.weights_dec = [1 / sum(self.eval_ortho(l, x) ** 2 for l in range(Q)) for x in nodes]
        self.nodes = np.array([float(x) for x in nodes])
        self.weights = np.array([float(w) for w in self.weights_dec])

    def _eval_monic_with_derivative(self, Q, x):
        p0, p1 = Decimal(1), x - self.alpha[0]
        d0, d1 = Decimal(0), Decimal(1)
        if Q == 0:
            return p0, d0
        for l in range(1, Q):
            p2 = (x - self.alpha[l]) * p1 - self.beta[l] * p0
            d2 = p1 + (x - self.alpha[l]) * d1 - self.beta[l] * d0
            p0, p1, d0, d1 = p1, p2, d1, d2
        return p1, d1

    def eval_ortho(self, l: int, x: Decimal) -> Decimal:
        """Orthonormal polynomial h_l at x (Horner on its decimal coefficients, at the rule's
        working precision)."""
        with localcontext() as c:
            c.prec = self.prec
            r = Decimal(0)
            for co in reversed(self.ortho[l]):
                r = r * x + co
            return +r


@functools.lru_cache(maxsize=None)
def half_range_rule(Q: int) -> GaussRule:
    """Half-range Gauss-Hermite rule of order Q on [0, inf) (Sec. III A 2)."""
    return GaussRule(Q, half_range_moment)


@functools.lru_cache(maxsize=None)
def full_range_rule(Q: int) -> GaussRule:
    """Full-range Gauss-Hermite rule of order Q on R (App. A)."""
    return GaussRule(Q, full_range_moment)


def lagrange_basis(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """l_k(x) = prod_{j != k} (x - p_j)/(p_k - p_j); returns [len(nodes), *x.shape]."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones((len(nodes),) + x.shape)
    for k in range(len(nodes)):
        for j in range(len(nodes)):
            if j != k:
                out[k] *= (x - nodes[j]) / (nodes[k] - nodes[j])
    return out


# Order of the auxiliary rules used to evaluate the projection integrals.
# Full line: the integrand is polynomial x Gaussian after the change of variable,
# so the auxiliary Gauss-Hermite rule is exact once 2M > degree.  Half line: the
# integrand is polynomial x omega(q) x exp(q v - v^2/2); with 2M >= Q + 60 (Q the
# order projected on) the rule integrates the polynomial of degree Q + 2 times the
# exponential's Taylor series far past the float64 round-off for |v| <= 1/2: 40
# points up to Q = 20, Q/2 + 30 above.
AUX_HALF = 40
AUX_FULL = 24


def project_half(nodes: np.ndarray, u, T, amax: int = 3) -> np.ndarray:
    """Discrete values on the positive half-axis of h_a(p) = (p-u)^a g(p; u, T).

    g(p; u, T) = exp(-(p-u)^2/(2T))/sqrt(2 pi T) is the unit-density 1D
    Maxwellian.  value[a, k, ...] = int_0^inf l_k(p) (p-u)^a g(p; u, T) dp,
    which is the truncated half-range expansion (Sec. III A 2, Eq. (hh_gk)).
    Evaluated with p = sqrt(T) q, which turns g sqrt(T) dq into
    omega(q) exp(q v - v^2/2) dq with v = u/sqrt(T), and a half-range Gauss rule
    in q of max(AUX_HALF, Q/2 + 30) points.  u, T broadcast (arrays over grid nodes).

    The negative half-axis value at node -p_k is (-1)^a project_half(nodes, -u, T)[a, k]
    (substitute p -> -p)."""
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    aux = half_range_rule(max(AUX_HALF, len(nodes) // 2 + 30))
    q = aux.nodes.reshape((-1,) + (1,) * u.ndim)
    W = aux.weights.reshape((-1,) + (1,) * u.ndim)
    v = u / np.sqrt(T)
    x = np.sqrt(T) * q                        # physical momentum at aux node
    E = W * np.exp(q * v - 0.5 * v * v)       # weight x non-polynomial factor
    L = lagrange_basis(nodes, x)              # [Q, M, ...]
    out = np.empty((amax + 1, len(nodes)) + np.broadcast(u, T).shape)
    for a in range(amax + 1):
        out[a] = np.sum(L * (E * (x - u) ** a)[None], axis=1)
    return out


def project_full(nodes: np.ndarray, u, T, amax: int = 3) -> np.ndarray:
    """Discrete values on the full axis of (p-u)^a g(p; u, T) (App. A, Eq. (H_gk)).

    value[a, k, ...] = int_R l_k(p) (p-u)^a g(p; u, T) dp, evaluated exactly with
    p = u + sqrt(T) y and an AUX_FULL-point Gauss-Hermite rule in y."""
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    # the integrand is a polynomial of degree len(nodes) - 1 + amax times the rule's weight:
    # exact once 2 M - 1 reaches that degree (AUX_FULL points at least)
    aux = full_range_rule(max(AUX_FULL, (len(nodes) + amax) // 2 + 1))
    y = aux.nodes.reshape((-1,) + (1,) * u.ndim)
    W = aux.weights.reshape((-1,) + (1,) * u.ndim)
    x = u + np.sqrt(T) * y
    L = lagrange_basis(nodes, x)
    out = np.empty((amax + 1, len(nodes)) + np.broadcast(u, T).shape)
    for a in range(amax + 1):
        out[a] = np.sum(L * (W * (np.sqrt(T) * y) ** a)[None], axis=1)
    return out


def force_matrix(Q: int) -> np.ndarray:
    """Momentum-derivative kernel on a full-range axis (App. A, Eq. (kernel_H)).

    K[k, k'] = -w_k sum_{l=0}^{Q-2} He_{l+1}(p_k) He_l(p_k') / l!  (p_0 = 1), so that
    (d f/d p)_k = sum_k' K[k, k'] f_k'.  He_l are the probabilists' Hermite
    polynomials, evaluated by He_{l+1} = p He_l - l He_{l-1}."""
    rule = full_range_rule(Q)
    p, w = rule.nodes, rule.weights
    He = np.zeros((Q + 1, Q))
    He[0] = 1.0
    if Q > 0:
        He[1] = p
    for l in range(1, Q):
        He[l + 1] = p * He[l] - l * He[l - 1]
    K = np.zeros((Q, Q))
    for l in range(Q - 1):
        K -= np.outer(w * He[l + 1], He[l]) / math.factorial(l)
    return K
