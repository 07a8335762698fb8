"""Pins of the oracle's time integrator (Eq. rk3) and WENO-5 smoothness indicators
(Eq. weno5_sigma) against what the mathematics fixes, independently of the oracle's own
formulas.

RK3: on a spatially uniform state the flux differences vanish at nodes far from the walls,
and a deviation d from the local equilibrium that leaves n, u, T and q unchanged relaxes
linearly, dd/dt = -d/tau.  One step of a Runge-Kutta method multiplies d by its stability
polynomial R(z), z = dt/tau; for the three-stage third-order scheme of Eq. (rk3) that is the
cubic Taylor polynomial of exp(-z), 1 - z + z^2/2 - z^3/6 (third order forces it).  A swapped
or mistyped stage weight changes R at first or second order in z.

WENO-5: the indicators of Eq. (weno5_sigma) are those of Jiang & Shu (J. Comput. Phys. 126,
1996): beta_q = sum_{l=1,2} h^(2l-1) int_cell (d^l P_q/dx^l)^2 dx, where P_q is the quadratic
whose averages over the three cells of candidate stencil q equal the three node values
(finite-difference WENO reconstructs the flux as cell averages of a primitive function).  The
candidate face values of Sec. III B 2 are P_q at the right face.  Both are computed here
exactly in rational arithmetic from that definition.
"""
import os
import random
from fractions import Fraction

import numpy as np

from oracle import fdlb as ofd
from oracle import quadrature as qd

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


# ----------------------------------------------------------------------------- RK3

def poly_mul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def poly_add(*ps):
    n = max(len(p) for p in ps)
    out = [Fraction(0)] * n
    for p in ps:
        for i, x in enumerate(p):
            out[i] += x
    return out


def poly_scale(p, c):
    return [c * x for x in p]


def stability_polynomial(stage2, stage3):
    """R(z) of the Shu-Osher scheme f1 = f + dt L(f); f2 = a f + b f1 + c dt L(f1);
    f_new = a' f + b' f2 + c' dt L(f2), applied to L(f) = -f/tau (coefficients in powers of z)."""
    one = [Fraction(1)]
    mz = [Fraction(0), Fraction(-1)]                       # -z
    d1 = poly_add(one, mz)                                 # 1 - z
    a, b, c = stage2
    d2 = poly_add(poly_scale(one, a), poly_scale(d1, b), poly_scale(poly_mul(mz, d1), c))
    a, b, c = stage3
    return poly_add(poly_scale(one, a), poly_scale(d2, b), poly_scale(poly_mul(mz, d2), c))


def test_golden_rk3_weights_are_third_order():
    """The printed stage weights of Eq. (rk3) compose to the cubic Taylor polynomial of e^-z."""
    g = golden()
    R = stability_polynomial(g["rk3_stage2"], g["rk3_stage3"])
    assert R == [Fraction(1), Fraction(-1), Fraction(1, 2), Fraction(-1, 6)]
    # and a swap of the stage-2 weights would not be
    s2 = g["rk3_stage2"]
    assert stability_polynomial([s2[1], s2[0], s2[2]], g["rk3_stage3"]) != R


def _uniform_deviation_case(z_target):
    """1D reduced Fourier set-up with equal wall temperatures, a uniform state f_eq + d with
    d_phi = eps w (p^2 - 1), d_theta = -2 eps w (zero change of n, n u, energy and q), and
    dt = z_target tau."""
    Q, N = 4, 64
    base = ofd.Params(nx=N, qx_half=Q, qy=0, qz=0, kn=0.02, eta0=0.1, T_left=1.0, T_right=1.0)
    o = ofd.Oracle(base)
    M = o.moments()
    tau = float(o.nodal(M)["tau"][N // 2])
    prm = ofd.Params(nx=N, qx_half=Q, qy=0, qz=0, kn=0.02, eta0=0.1, T_left=1.0, T_right=1.0,
                     dt=z_target * tau)
    o = ofd.Oracle(prm)
    rule = qd.half_range_rule(Q)
    p = np.concatenate([rule.nodes, -rule.nodes])
    w = np.concatenate([rule.weights, rule.weights])      # each half-line carries half the mass
    eps = 1e-3
    feq = o.f.copy()
    d = np.zeros_like(feq)
    d[:, 0, :] = (eps * w * (p * p - 1.0))[:, None]
    d[:, 1, :] = (-2.0 * eps * w)[:, None]
    o.f = feq + d
    return o, feq, d, tau


def test_rk3_step_multiplies_relaxing_deviation_by_stability_polynomial():
    """One oracle step multiplies the deviation at central nodes by 1 - z + z^2/2 - z^3/6."""
    for z_target in (0.3, 0.8):
        o, feq, d, tau = _uniform_deviation_case(z_target)
        # the deviation changes neither n, u, T nor q: the moments are those of f_eq
        M, M0 = o.moments(), o.moments(feq)
        for key in ("n", "ux", "T", "qx"):
            np.testing.assert_allclose(M[key], M0[key], rtol=0, atol=1e-14)
        tau_now = o.nodal(M)["tau"]
        z = o.dt / tau_now
        o.step(1)
        centre = slice(24, 40)                  # 24 nodes from each wall: beyond the walls' reach in one step
        R = 1.0 - z + z * z / 2.0 - z ** 3 / 6.0
        dev = o.f[:, :, centre] - feq[:, :, centre]
        expect = R[None, None, centre] * d[:, :, centre]
        np.testing.assert_allclose(dev, expect, rtol=1e-11, atol=1e-16)
        assert abs(float(z[32]) - z_target) < 1e-12


# ----------------------------------------------------------------------------- WENO-5

def quadratic_from_averages(values, cells):
    """Coefficients (c0, c1, c2) of P(x) = c0 + c1 x + c2 x^2 whose average over the unit cell
    [j - 1/2, j + 1/2] is values[m] for j = cells[m] (exact rational solve)."""
    rows = []
    for j in cells:
        a, b = Fraction(2 * j - 1, 2), Fraction(2 * j + 1, 2)
        # average of x^k over [a, b] (width 1)
        rows.append([(b ** (k + 1) - a ** (k + 1)) / (k + 1) for k in range(3)])
    A = [r[:] + [Fraction(v)] for r, v in zip(rows, values)]
    for col in range(3):                      # Gauss-Jordan on the 3 x 3 system
        piv = next(r for r in range(col, 3) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        inv = 1 / A[col][col]
        A[col] = [x * inv for x in A[col]]
        for r in range(3):
            if r != col and A[r][col] != 0:
                fac = A[r][col]
                A[r] = [x - fac * y for x, y in zip(A[r], A[col])]
    return [A[k][3] for k in range(3)]


def jiang_shu_beta(c):
    """sum_{l=1,2} int_{-1/2}^{1/2} (d^l P/dx^l)^2 dx for P = c0 + c1 x + c2 x^2 (h = 1)."""
    c0, c1, c2 = c
    # P' = c1 + 2 c2 x: int P'^2 = c1^2 + (4 c2^2)/12 (the odd term integrates to zero)
    first = c1 * c1 + Fraction(4, 12) * c2 * c2
    second = (2 * c2) ** 2
    return first + second


STENCILS = ((-2, -1, 0), (-1, 0, 1), (0, 1, 2))


def test_weno_indicators_from_jiang_shu_definition():
    rng = random.Random(2308)
    for _ in range(200):
        v = [rng.uniform(-2.0, 2.0) for _ in range(5)]      # f_{i-2} .. f_{i+2}
        exact = []
        faces = []
        for cells in STENCILS:
            vals = [Fraction(v[j + 2]) for j in cells]
            c = quadratic_from_averages(vals, cells)
            exact.append(jiang_shu_beta(c))
            faces.append(c[0] + c[1] * Fraction(1, 2) + c[2] * Fraction(1, 4))
        got = ofd.weno5_indicators(*[np.float64(x) for x in v])
        scale = max(float(abs(e)) for e in exact) + 1e-300
        for g_, e in zip(got, exact):
            assert abs(float(g_) - float(e)) <= 1e-14 * scale
        cand = ofd.weno5_candidates(*[np.float64(x) for x in v])
        for g_, e in zip(cand, faces):
            assert abs(float(g_) - float(e)) <= 1e-14 * (1 + abs(float(e)))


def test_weno_indicator_constants_are_not_free():
    """A change of 13/12 or 1/4 in the indicators departs from the definition on generic data."""
    v = [Fraction(x) for x in (3, -1, 4, 1, -5)]
    c = quadratic_from_averages(v[0:3], STENCILS[0])
    beta = jiang_shu_beta(c)
    t1 = v[0] - 2 * v[1] + v[2]
    t2 = v[0] - 4 * v[1] + 3 * v[2]
    assert beta == Fraction(13, 12) * t1 ** 2 + Fraction(1, 4) * t2 ** 2
    assert beta != Fraction(12, 13) * t1 ** 2 + Fraction(1, 4) * t2 ** 2
    assert beta != Fraction(13, 12) * t1 ** 2 + Fraction(1, 2) * t2 ** 2
