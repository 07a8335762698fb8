"""Plain FP64 CPU oracle of the FDLB solver for the simplified Enskog equation.

Test infrastructure only (see ``oracle/__init__``).  Numpy arrays, no blocking,
fusion or reordering beyond what the equations state.  Layout: f[kx, t, i]
with kx over the 2 Q_x^h x-velocities (+p_1..+p_Q, then -p_1..-p_Q), t over
the transverse velocity index, i over the N grid nodes.

One RK3 stage computes, in the paper's order:
  moments (Eq. macro_LB; the Eq. macro2D/macro1D forms for reduced slots),
  chi_SET (Eq. chi), Pr (Eq. prandtl), mu (Eq. viscosity), tau (Eq. tau),
  6th-order gradients (Sec. III B 3), the Shakhov target (Eqs. j0 and the f^S
  formula of Sec. II A) plus tau J1 (Eq. j1), the diffuse-reflection closure
  (Sec. III B), WENO-5 fluxes (Eqs. weno5_flux_x .. weno5_sigma), the force term
  (App. A, Eq. kernel_H) and the TVD RK3 combination (Eq. rk3).

Readings where the paper is silent, garbled or ambiguous (each restated where it
is used):
  R1  Units: m = k_B = T_ref = 1, channel width D = 1, mean density n0 = 1,
      so b n = 4 eta and eta_i = eta0 n_i (Eq. chi and the eta definition below
      it).  Kn refers to D:  mu0(T) = (5/16) sqrt(2 pi) chi(eta0) Kn sqrt(T)
      (Kn definition of Sec. II A combined with mu0).
  R2  The discrete equilibrium is the truncated expansion (order Q-1 on each
      half-axis / axis), i.e. the projection that reproduces the first Q
      moments; f^S and tau J1 are projected monomial by monomial.
  R3  J1 is the 3D form Eq. (j1) with zeta = xi/sqrt(2T); the reduced forms
      follow by integrating over p_z (and p_y).  This reproduces Eqs.
      (j1_expanded_1D)/(j1_expanded_2D) with the d_x u_x coefficient read as
      3/5 (1D, phi) and the theta_2D prefactor read as k_B T (not 2 m k_B T).
      The shear term 2 zeta_x zeta_y d_x u_y, absent from Eq. (j1_expanded_2D),
      is off by default (``j1_shear=False``) and on with ``j1_shear=True``.
  R4  Gradients of ln n, ln chi, ln T, u_x, u_y (J1 needs d ln chi; Sec. III B 3
      lists ln rho, u, ln T), 6th order central in the mapped coordinate s,
      one-sided / biased 7-point stencils (Fornberg) at the 3 nodes next to
      each wall.
  R5  Grid: cell-centred nodes s_i = -1 + (i + 1/2) ds, ds = 2/N, x(s) uniform
      (x = s/2) or tanh-stretched x = tanh(A s)/(2 tanh A); walls at the cell
      faces s = +-1.  Advection in s: -(p_x/(x'(s_i) ds)) (F_{i+1/2} - F_{i-1/2}).
  R6  Diffuse walls: outgoing populations get quadratically extrapolated
      ghosts; the wall-face flux of outgoing populations is the quadratic
      reconstruction p (11 f_1 - 7 f_2 + 2 f_3)/6 (what all three WENO candidates
      give with those ghosts); n_w makes the net mass flux through the wall
      zero; incoming populations get ghosts and wall-face flux n_w g_wall.
  R7  WENO weights without epsilon: omega~_q = delta_q/phi_q^2.  When some
      phi_q == 0 the weights are delta_q / sum_{r: phi_r = 0} delta_r on the
      vanishing set and 0 elsewhere (the limit phi -> 0).  Otherwise the
      normalised weights are computed as delta_q (phi_min/phi_q)^2 / sum, which
      equals delta_q/phi_q^2 / sum exactly in real arithmetic and cannot
      overflow.  For p_x < 0 the stencil is mirrored about the face.
  R8  Force: L contains -a_y (d f/d p_y) (the printed Eq. cast drops -F_y;
      Eq. evolution_2D has it).
  R9  Residual per step: max of ||n^n - n^{n-1}|| / ||n^n||, ||T^n - T^{n-1}|| /
      ||T^n||, ||u_x^n - u_x^{n-1}||, ||u_y^n - u_y^{n-1}|| with the cell-width
      weighted L2 norm ||v|| = sqrt(sum_i x'_i ds v_i^2).
  R10 Time step dt = CFL min_i(x'(s_i) ds) / max_k p_k unless given.
  R15 chi_RET-FM (Eq. chi_ret): chi_SET of the density averaged over a ball of radius
      sigma = 6 sqrt(2) eta0 chi(eta0) Kn (the Kn definition of Sec. II A with n0 = D = 1),
      evaluated at the node; b rho in the closure stays the local 4 eta0 n.  In the
      channel n depends on x only, is constant on each grid cell and zero beyond the
      walls, which reduces the ball average to a 1D average with weight
      3 (sigma^2 - t^2)/(4 sigma^3), integrated exactly over each cell.
  R16 Full-range x quadrature (App. A; the comparison of its last figure): the
      full-range Gauss-Hermite rule of even order 2 Q_x^h replaces the two
      half-range rules, so the x-velocities keep the form {+p_k} u {-p_k} (an
      odd order would add a zero node, which this layout does not hold).  The
      discrete equilibrium is one expansion over the whole axis truncated at
      order 2 Q_x^h - 1 (Eq. H_gk); walls, fluxes and moments are unchanged.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from . import quadrature as qd

FOURIER, COUETTE, POISEUILLE = 0, 1, 2


@dataclass
class Params:
    """Solver parameters (same meaning as the C-ABI ``fdlb_params``)."""
    nx: int
    qx_half: int
    qy: int                 # 0 -> p_y integrated out too (1D reduced, Sec. II B 1)
    qz: int                 # 0 -> p_z integrated out: (phi, theta) slots (Sec. II B)
    kn: float
    eta0: float
    T_left: float = 1.0
    T_right: float = 1.0
    U_left: float = 0.0
    U_right: float = 0.0
    accel_y: float = 0.0
    grid: str = "uniform"   # or "tanh"
    stretch: float = 1.5
    cfl: float = 0.5
    dt: float = 0.0         # 0 -> from cfl (R10)
    j1_shear: bool = False
    flow: int = FOURIER
    T_init: float = 0.0     # 0 -> mean wall temperature
    chi_model: str = "set"  # "set": chi_SET[n]; "ret-fm": chi_SET[n-bar] (Eq. chi_ret, R15)
    x_quadrature: str = "half"  # "half": half-range order qx_half per side (Sec. III A 2);
                                # "full": full-range Gauss-Hermite order 2 qx_half (App. A)


# ----------------------------------------------------------------------------
# Closed forms of Sec. II
# ----------------------------------------------------------------------------

def chi_set(eta):
    """Carnahan-Starling contact value, Eq. (chi): (2 - eta) / (2 (1 - eta)^3)."""
    eta = np.asarray(eta, dtype=np.float64)
    return (2.0 - eta) / (2.0 * (1.0 - eta) ** 3)


def eos_ratio(eta):
    """P^hs/(n k_B T) of Eq. (eos): (1 + eta + eta^2 - eta^3)/(1 - eta)^3."""
    eta = np.asarray(eta, dtype=np.float64)
    return (1.0 + eta + eta ** 2 - eta ** 3) / (1.0 - eta) ** 3


def prandtl(brc):
    """Dense-gas Prandtl number, Eq. (prandtl), as a function of b rho chi."""
    brc = np.asarray(brc, dtype=np.float64)
    num = 1.0 + 0.8 * brc + (4.0 / 25.0) * (1.0 + 12.0 / math.pi) * brc ** 2
    den = 1.0 + 1.2 * brc + (9.0 / 25.0) * (1.0 + 32.0 / (9.0 * math.pi)) * brc ** 2
    return (2.0 / 3.0) * num / den


def mu0(T, kn, eta0):
    """Hard-sphere viscosity mu0 = 5/(16 sigma^2) sqrt(T/pi) with sigma fixed by Kn (R1)."""
    return (5.0 / 16.0) * math.sqrt(2.0 * math.pi) * float(chi_set(eta0)) * kn * np.sqrt(T)


def viscosity(n, T, kn, eta0, chi=None):
    """Enskog shear viscosity, Eq. (viscosity): mu0 [1/chi + 4/5 b rho + 4/25 (1 + 12/pi)(b rho)^2 chi]
    (chi = chi_SET[n] unless given)."""
    eta = eta0 * np.asarray(n, dtype=np.float64)
    chi = chi_set(eta) if chi is None else chi
    br = 4.0 * eta
    return mu0(T, kn, eta0) * (1.0 / chi + 0.8 * br + (4.0 / 25.0) * (1.0 + 12.0 / math.pi) * br ** 2 * chi)


def sphere_diameter(eta0, kn):
    """Molecular diameter in units of the channel width: Kn = 1/(sqrt(2) pi sigma^2 n0 chi0 D)
    with b n0 = 4 eta0 and b = 2 pi sigma^3/3 gives sigma = 6 sqrt(2) eta0 chi(eta0) Kn (R1)."""
    return 6.0 * math.sqrt(2.0) * eta0 * float(chi_set(eta0)) * kn


def ret_fm_weights(faces, nodes, sigma):
    """Averaging matrix of the Fischer-Methfessel density (Eq. chi_ret and the definition of
    n-bar below it) in a channel, reading R15: n depends on x only and is constant on each
    cell [faces[j], faces[j+1]], zero outside the walls.  The ball average then reduces to
    n-bar(x_i) = 3/(4 sigma^3) int n(x_i + t) (sigma^2 - t^2) dt over |t| < sigma, so
    W[i, j] = 3/(4 sigma^3) int of (sigma^2 - t^2) over the part of cell j within the window."""
    K = lambda t: sigma * sigma * t - t ** 3 / 3.0
    lo = np.clip(np.asarray(faces[:-1])[None, :] - np.asarray(nodes)[:, None], -sigma, sigma)
    hi = np.clip(np.asarray(faces[1:])[None, :] - np.asarray(nodes)[:, None], -sigma, sigma)
    return 3.0 / (4.0 * sigma ** 3) * (K(hi) - K(lo))


def knudsen(eta0, R):
    """Kn of Sec. II A in terms of the confinement ratio: 1/(6 sqrt(2) eta0 chi(eta0) R)."""
    return 1.0 / (6.0 * math.sqrt(2.0) * eta0 * float(chi_set(eta0)) * R)


# ----------------------------------------------------------------------------
# Finite-difference weights (Fornberg's construction, done exactly)
# ----------------------------------------------------------------------------

def fd_weights(offsets, x0, deriv=1):
    """Exact rational weights c_j with sum_j c_j F(offsets_j) = F^(deriv)(x0) for
    polynomials F of degree < len(offsets) (solves the moment system in Fractions)."""
    n = len(offsets)
    A = [[Fraction(o - x0) ** r for o in offsets] for r in range(n)]
    b = [Fraction(0)] * n
    b[deriv] = Fraction(math.factorial(deriv))
    # Gaussian elimination in exact arithmetic.
    M = [row[:] + [b[r]] for r, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                fac = M[r][c] / M[c][c]
                M[r] = [a - fac * bb for a, bb in zip(M[r], M[c])]
    return [M[r][n] / M[r][r] for r in range(n)]


def gradient_matrix(N: int) -> np.ndarray:
    """D[i, j]: d/ds at node i from node values, 6th order (Sec. III B 3, R4).

    Interior nodes 3..N-4 use the central stencil of Sec. III B 3; nodes 0,1,2 use
    the 7-point stencils on nodes 0..6, mirrored at the right wall."""
    D = np.zeros((N, N))
    for i in range(N):
        if 3 <= i <= N - 4:
            nodes = list(range(i - 3, i + 4))
        elif i < 3:
            nodes = list(range(0, 7))
        else:
            nodes = list(range(N - 7, N))
        w = fd_weights(nodes, i)
        for j, c in zip(nodes, w):
            D[i, j] = float(c)
    return D


# ----------------------------------------------------------------------------
# WENO-5 (Sec. III B 2)
# ----------------------------------------------------------------------------

DELTA = (0.1, 0.6, 0.3)


def weno5_candidates(vm2, vm1, v0, vp1, vp2):
    """The three interpolating fluxes F^1, F^2, F^3 of Sec. III B 2 (per unit p/m)."""
    F1 = vm2 / 3.0 - 7.0 / 6.0 * vm1 + 11.0 / 6.0 * v0
    F2 = -vm1 / 6.0 + 5.0 / 6.0 * v0 + vp1 / 3.0
    F3 = v0 / 3.0 + 5.0 / 6.0 * vp1 - vp2 / 6.0
    return F1, F2, F3


def weno5_indicators(vm2, vm1, v0, vp1, vp2):
    """Smoothness indicators varphi_1..3 of Eq. (weno5_sigma)."""
    s1 = 13.0 / 12.0 * (vm2 - 2.0 * vm1 + v0) ** 2 + 0.25 * (vm2 - 4.0 * vm1 + 3.0 * v0) ** 2
    s2 = 13.0 / 12.0 * (vm1 - 2.0 * v0 + vp1) ** 2 + 0.25 * (vm1 - vp1) ** 2
    s3 = 13.0 / 12.0 * (v0 - 2.0 * vp1 + vp2) ** 2 + 0.25 * (3.0 * v0 - 4.0 * vp1 + vp2) ** 2
    return s1, s2, s3


def weno5_face(vm2, vm1, v0, vp1, vp2):
    """Upwind-biased face value of Eq. (weno5_flux_x) for a positive advection
    velocity, from the five node values f_{i-2..i+2} (face i+1/2), with the
    epsilon-free weights of Eq. (weno5_omega_x) and reading R7."""
    F1, F2, F3 = weno5_candidates(vm2, vm1, v0, vp1, vp2)
    s1, s2, s3 = weno5_indicators(vm2, vm1, v0, vp1, vp2)
    phi = np.stack([s1, s2, s3])
    zero = phi == 0.0
    anyzero = zero.any(axis=0)
    delta = np.array(DELTA).reshape((3,) + (1,) * s1.ndim)
    # limiting case: weight only on the vanishing indicators
    wz = np.where(zero, delta, 0.0)
    wz = wz / np.where(anyzero, wz.sum(axis=0), 1.0)
    # regular case: delta_q/phi_q^2, rescaled by phi_min^2 (evaluated everywhere; where an
    # indicator vanishes it may overflow, and the limiting case above is taken instead)
    pmin = np.where(anyzero, 1.0, phi.min(axis=0))
    safe = np.where(zero, 1.0, phi)
    with np.errstate(over="ignore", invalid="ignore"):
        wr = delta * (pmin / safe) ** 2
        wr = wr / wr.sum(axis=0)
    w = np.where(anyzero[None], wz, wr)
    return w[0] * F1 + w[1] * F2 + w[2] * F3


# ----------------------------------------------------------------------------
# The solver
# ----------------------------------------------------------------------------

# The 13 monomials xi_x^a xi_y^b xi_z^c of f^S and tau J1 (a <= 3, b <= 3, c in {0, 2}).
MONOMIALS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0),
             (3, 0, 0), (1, 2, 0), (1, 0, 2), (2, 1, 0), (0, 3, 0), (0, 1, 2)]


def gauss_moment(k: int, T):
    """E[xi^k] for a centred 1D Gaussian of variance T: (k-1)!! T^(k/2), 0 for odd k."""
    if k % 2:
        return np.zeros_like(np.asarray(T, dtype=np.float64))
    r = 1.0
    for j in range(1, k, 2):
        r *= j
    return r * np.asarray(T, dtype=np.float64) ** (k // 2)


class Oracle:
    """FDLB solver state for one instance (FP64)."""

    def __init__(self, prm: Params):
        self.prm = prm
        N = prm.nx
        if N < 8:
            raise ValueError("nx must be >= 8")
        if prm.qx_half < 1:
            raise ValueError("qx_half must be >= 1")
        if prm.qy == 0 and prm.qz != 0:
            raise ValueError("qy == 0 requires qz == 0 (1D reduced form)")
        if prm.qy == 0 and (prm.U_left or prm.U_right or prm.accel_y):
            raise ValueError("the 1D reduced form has no y dynamics")
        self.N = N
        Q = prm.qx_half
        self.Q = Q
        # x axis: half-range rule, discrete set {+p_k} then {-p_k} (Eq. hh_pk); or the
        # full-range rule of even order 2Q (App. A), whose nodes are the same kind of set
        # {+p_k} u {-p_k} (no zero node), stored in the same order
        if prm.x_quadrature == "half":
            self.xrule = qd.half_range_rule(Q)
            p = self.xrule.nodes
        elif prm.x_quadrature == "full":
            self.xrule = qd.full_range_rule(2 * Q)
            p = self.xrule.nodes[Q:]              # ascending: the positive half
        else:
            raise ValueError("x_quadrature must be 'half' or 'full'")
        self.px = np.concatenate([p, -p])
        # transverse axes
        if prm.qy > 0:
            self.yrule = qd.full_range_rule(prm.qy)
        if prm.qz > 0:
            self.zrule = qd.full_range_rule(prm.qz)
        if prm.qy > 0 and prm.qz > 0:
            self.form = "unreduced"
            y, z = self.yrule.nodes, self.zrule.nodes
            self.Tc = prm.qy * prm.qz
            self.mt = np.ones(self.Tc)
            self.py = np.repeat(y, prm.qz)
            self.et = np.tile(0.5 * z * z, prm.qy)
        elif prm.qy > 0:
            self.form = "reduced2d"
            self.Tc = prm.qy * 2
            self.mt = np.tile([1.0, 0.0], prm.qy)
            self.py = np.repeat(self.yrule.nodes, 2)
            self.et = np.tile([0.0, 0.5], prm.qy)
        else:
            self.form = "reduced1d"
            self.Tc = 2
            self.mt = np.array([1.0, 0.0])
            self.py = np.zeros(2)
            self.et = np.array([0.0, 0.5])
        # grid (R5)
        self.ds = 2.0 / N
        s = -1.0 + (np.arange(N) + 0.5) * self.ds
        if prm.grid == "uniform":
            self.x = 0.5 * s
            self.xp = np.full(N, 0.5)
        elif prm.grid == "tanh":
            A = prm.stretch
            self.x = 0.5 * np.tanh(A * s) / math.tanh(A)
            self.xp = 0.5 * A / (np.cosh(A * s) ** 2 * math.tanh(A))
        else:
            raise ValueError("grid must be 'uniform' or 'tanh'")
        self.dx = self.xp * self.ds
        sf = -1.0 + np.arange(N + 1) * self.ds                      # cell faces in s
        self.faces = 0.5 * sf if prm.grid == "uniform" else 0.5 * np.tanh(prm.stretch * sf) / math.tanh(prm.stretch)
        if prm.chi_model == "ret-fm":
            self.sigma = sphere_diameter(prm.eta0, prm.kn)
            self.Wfm = ret_fm_weights(self.faces, self.x, self.sigma)
        elif prm.chi_model != "set":
            raise ValueError("chi_model must be 'set' or 'ret-fm'")
        self.dt = prm.dt if prm.dt > 0 else prm.cfl * self.dx.min() / p.max()
        self.Dmat = gradient_matrix(N)
        self.chi0 = float(chi_set(prm.eta0))
        if self.form != "reduced1d":
            self.Ky = qd.force_matrix(prm.qy)
        # wall Maxwellians, unit density (R6)
        self.gL = self.equilibrium(np.ones(1), np.zeros(1), np.full(1, prm.U_left), np.full(1, prm.T_left))[..., 0]
        self.gR = self.equilibrium(np.ones(1), np.zeros(1), np.full(1, prm.U_right), np.full(1, prm.T_right))[..., 0]
        T0 = prm.T_init if prm.T_init > 0 else 0.5 * (prm.T_left + prm.T_right)
        self.f = self.equilibrium(np.ones(N), np.zeros(N), np.zeros(N), np.full(N, T0))
        self.steps = 0
        self.last_residual = math.inf
        self._prev_prim = None

    # -- velocity-space projections (R2) -----------------------------------
    def x_projection(self, ux, T):
        """P^x[a, kx, i]: projected (p_x - u_x)^a g(p_x; u_x, T) on the 2Q x-velocities."""
        if self.prm.x_quadrature == "full":
            # one expansion over the whole axis, truncated at order 2Q - 1 (App. A, Eq. H_gk)
            return qd.project_full(self.px, ux, T)
        p = self.xrule.nodes
        pos = qd.project_half(p, ux, T)
        neg = qd.project_half(p, -ux, T)
        sign = np.array([1.0, -1.0, 1.0, -1.0]).reshape(4, 1, 1)
        return np.concatenate([pos, sign * neg], axis=1)

    def transverse(self, coef, uy, T):
        """Y[a, t, i] = sum over monomials (a, b, c) of coef * (y,z)-factor at t."""
        Y = np.zeros((4, self.Tc) + np.shape(T))
        if self.form == "reduced1d":
            for (a, b, c), cv in coef.items():
                phi = gauss_moment(b, T) * gauss_moment(c, T)
                theta = gauss_moment(b + 2, T) * gauss_moment(c, T) + gauss_moment(b, T) * gauss_moment(c + 2, T)
                Y[a, 0] += cv * phi
                Y[a, 1] += cv * theta
            return Y
        Py = qd.project_full(self.yrule.nodes, uy, T)            # [b, ky, i]
        if self.form == "unreduced":
            Pz = qd.project_full(self.zrule.nodes, np.zeros_like(T), T)   # [c, kz, i]
            for (a, b, c), cv in coef.items():
                Y[a] += cv * (Py[b][:, None] * Pz[c][None, :]).reshape((self.Tc,) + np.shape(T))
        else:
            for (a, b, c), cv in coef.items():
                zf = np.stack([gauss_moment(c, T), gauss_moment(c + 2, T)])     # phi, theta slots
                Y[a] += cv * (Py[b][:, None] * zf[None, :]).reshape((self.Tc,) + np.shape(T))
        return Y

    def assemble(self, n, ux, uy, T, coef):
        """Discrete values n * sum_a P^x_a[kx] Y_a[t] of n g(xi) sum coef xi^(a,b,c)."""
        Px = self.x_projection(ux, T)
        Y = self.transverse(coef, uy, T)
        return n * np.einsum("aki,ati->kti", Px, Y)

    def equilibrium(self, n, ux, uy, T):
        """Projected local Maxwellian (Sec. III A 2 and App. A discrete equilibria)."""
        return self.assemble(n, ux, uy, T, {(0, 0, 0): np.ones_like(T)})

    # -- moments (Eq. macro_LB) ---------------------------------------------
    def moments(self, f=None):
        """Returns dict of n, ux, uy, T, qx, qy, Pxx, Pxy (two-pass peculiar form)."""
        f = self.f if f is None else f
        px = self.px[:, None, None]
        py = self.py[None, :, None]
        mt = self.mt[None, :, None]
        et = self.et[None, :, None]
        n = np.sum(mt * f, axis=(0, 1))
        ux = np.sum(mt * px * f, axis=(0, 1)) / n
        uy = np.sum(mt * py * f, axis=(0, 1)) / n
        xx = px - ux[None, None, :]
        xy = py - uy[None, None, :]
        E = mt * 0.5 * (xx ** 2 + xy ** 2) + et
        T = np.sum(E * f, axis=(0, 1)) / (1.5 * n)
        qx = np.sum(xx * E * f, axis=(0, 1))
        qy = np.sum(xy * E * f, axis=(0, 1))
        Pxx = np.sum(mt * xx * xx * f, axis=(0, 1))
        Pxy = np.sum(mt * xx * xy * f, axis=(0, 1))
        return dict(n=n, ux=ux, uy=uy, T=T, qx=qx, qy=qy, Pxx=Pxx, Pxy=Pxy)

    # -- per-node closure ------------------------------------------------------
    def nodal(self, M):
        """chi, b rho chi, Pr, tau and the gradients G, B, U, V (R1, R4)."""
        prm = self.prm
        n, T = M["n"], M["T"]
        eta = prm.eta0 * n
        chi = chi_set(prm.eta0 * (self.Wfm @ n)) if prm.chi_model == "ret-fm" else chi_set(eta)
        brc = 4.0 * eta * chi
        Pr = prandtl(brc)
        tau = viscosity(n, T, prm.kn, prm.eta0, chi) / (n * T)
        d = lambda q: (self.Dmat @ q) / (self.xp * self.ds)
        G = 2.0 * d(np.log(n)) + d(np.log(chi)) + d(np.log(T))
        B = d(np.log(T))
        U = d(M["ux"])
        V = d(M["uy"])
        return dict(chi=chi, brc=brc, Pr=Pr, tau=tau, G=G, B=B, U=U, V=V)

    def target_coefficients(self, M, C):
        """Coefficients of the 13 monomials in f^S + tau J1 = n g(xi) * sum coef xi^(a,b,c).

        f^S: Shakhov factor 1 + (1 - Pr)/(5 n T^2) (|xi|^2/T - 5) xi.q (Sec. II A).
        tau J1: -tau b rho chi {xi_x [G + 3/5 (|xi|^2/(2T) - 5/2) B]
                + 2/5 [(xi_x^2/T) U + (|xi|^2/(2T) - 5/2) U] + shear 2/5 (xi_x xi_y/T) V}
        with G = d ln(n^2 chi T), B = d ln T, U = d u_x, V = d u_y (Eq. j1, R3)."""
        n, T, qx, qy = M["n"], M["T"], M["qx"], M["qy"]
        A = (1.0 - C["Pr"]) / (5.0 * n * T * T)
        W = -C["tau"] * C["brc"]
        G, B, U, V = C["G"], C["B"], C["U"], C["V"]
        sh = 1.0 if self.prm.j1_shear else 0.0
        c3 = A * qx / T + W * 0.3 * B / T
        cy = A * qy / T
        return {
            (0, 0, 0): 1.0 - W * U,
            (1, 0, 0): -5.0 * A * qx + W * (G - 1.5 * B),
            (0, 1, 0): -5.0 * A * qy,
            (2, 0, 0): W * 0.6 * U / T,
            (0, 2, 0): W * 0.2 * U / T,
            (0, 0, 2): W * 0.2 * U / T,
            (1, 1, 0): W * sh * 0.4 * V / T,
            (3, 0, 0): c3, (1, 2, 0): c3, (1, 0, 2): c3,
            (2, 1, 0): cy, (0, 3, 0): cy, (0, 1, 2): cy,
        }

    def target(self, M, C):
        """Discrete f^S + tau J1 at every (kx, t, i)."""
        return self.assemble(M["n"], M["ux"], M["uy"], M["T"], self.target_coefficients(M, C))

    # -- wall closure and advection (R6, R7) --------------------------------------
    def wall_density(self, f):
        """(n_w^L, n_w^R): zero net mass flux through each wall."""
        Q = self.Q
        px = self.px[:, None]
        mt = self.mt[None, :]
        fhatL = (11.0 * f[..., 0] - 7.0 * f[..., 1] + 2.0 * f[..., 2]) / 6.0
        fhatR = (11.0 * f[..., -1] - 7.0 * f[..., -2] + 2.0 * f[..., -3]) / 6.0
        outL = np.sum((mt * px * fhatL)[Q:])          # p_x < 0 leaves through the left wall
        inL = np.sum((mt * px * self.gL)[:Q])
        outR = np.sum((mt * px * fhatR)[:Q])          # p_x > 0 leaves through the right wall
        inR = np.sum((mt * px * self.gR)[Q:])
        return -outL / inL, -outR / inR

    def advection(self, f, nwL, nwR):
        """-(p_x / (x' ds)) (F_{i+1/2} - F_{i-1/2}) with WENO-5 interior faces."""
        Q, N = self.Q, self.N
        g = np.zeros(f.shape[:2] + (N + 4,))
        g[..., 2:N + 2] = f
        # ghosts: index j = i + 2
        g[:Q, :, 0] = nwL * self.gL[:Q]
        g[:Q, :, 1] = nwL * self.gL[:Q]
        g[Q:, :, 1] = 3 * f[Q:, :, 0] - 3 * f[Q:, :, 1] + f[Q:, :, 2]
        g[Q:, :, 0] = 6 * f[Q:, :, 0] - 8 * f[Q:, :, 1] + 3 * f[Q:, :, 2]
        g[Q:, :, N + 2] = nwR * self.gR[Q:]
        g[Q:, :, N + 3] = nwR * self.gR[Q:]
        g[:Q, :, N + 2] = 3 * f[:Q, :, N - 1] - 3 * f[:Q, :, N - 2] + f[:Q, :, N - 3]
        g[:Q, :, N + 3] = 6 * f[:Q, :, N - 1] - 8 * f[:Q, :, N - 2] + 3 * f[:Q, :, N - 3]
        face = np.zeros(f.shape[:2] + (N + 1,))      # face j between nodes j-1 and j
        fi = np.arange(1, N)                          # interior faces
        # p > 0: stencil nodes j-3 .. j+1 -> g indices j-1 .. j+3
        face[:Q, :, 1:N] = weno5_face(g[:Q, :, fi - 1], g[:Q, :, fi], g[:Q, :, fi + 1], g[:Q, :, fi + 2], g[:Q, :, fi + 3])
        # p < 0: mirrored, nodes j+2 .. j-2 -> g indices j+4 .. j
        face[Q:, :, 1:N] = weno5_face(g[Q:, :, fi + 4], g[Q:, :, fi + 3], g[Q:, :, fi + 2], g[Q:, :, fi + 1], g[Q:, :, fi])
        # wall faces (R6)
        face[:Q, :, 0] = nwL * self.gL[:Q]
        face[Q:, :, 0] = (11.0 * f[Q:, :, 0] - 7.0 * f[Q:, :, 1] + 2.0 * f[Q:, :, 2]) / 6.0
        face[Q:, :, N] = nwR * self.gR[Q:]
        face[:Q, :, N] = (11.0 * f[:Q, :, N - 1] - 7.0 * f[:Q, :, N - 2] + 2.0 * f[:Q, :, N - 3]) / 6.0
        flux = self.px[:, None, None] * face
        return -(flux[..., 1:] - flux[..., :-1]) / (self.xp * self.ds)

    def force(self, f):
        """-a_y (d f / d p_y) with the kernel of App. A (R8)."""
        if self.form == "reduced1d" or self.prm.accel_y == 0.0:
            return np.zeros_like(f)
        Qy = self.prm.qy
        fs = f.reshape(f.shape[0], Qy, -1, f.shape[2])          # [kx, ky, kz|slot, i]
        d = np.einsum("yk,xkzi->xyzi", self.Ky, fs)
        return (-self.prm.accel_y * d).reshape(f.shape)

    def L(self, f):
        """Right-hand side of Eq. (cast)."""
        M = self.moments(f)
        C = self.nodal(M)
        nwL, nwR = self.wall_density(f)
        tgt = self.target(M, C)
        return self.advection(f, nwL, nwR) + self.force(f) - (f - tgt) / C["tau"][None, None, :]

    def step(self, nsteps: int = 1):
        """TVD RK3, Eq. (rk3), with the per-step residual (R9)."""
        dt = self.dt
        for _ in range(nsteps):
            f = self.f
            prev = self.primitive(f)
            f1 = f + dt * self.L(f)
            f2 = 0.75 * f + 0.25 * f1 + 0.25 * dt * self.L(f1)
            self.f = f / 3.0 + 2.0 / 3.0 * f2 + 2.0 / 3.0 * dt * self.L(f2)
            self.steps += 1
            self.last_residual = self.residual_between(prev, self.primitive(self.f))
        return self

    # -- diagnostics -----------------------------------------------------------
    def primitive(self, f=None):
        M = self.moments(f)
        return M["n"], M["ux"], M["uy"], M["T"]

    def norm(self, v):
        return math.sqrt(float(np.sum(self.dx * v * v)))

    def residual_between(self, old, new):
        (n0, ux0, uy0, T0), (n1, ux1, uy1, T1) = old, new
        return max(self.norm(n1 - n0) / self.norm(n1), self.norm(T1 - T0) / self.norm(T1),
                   self.norm(ux1 - ux0), self.norm(uy1 - uy0))

    def mass(self, f=None):
        f = self.f if f is None else f
        return float(np.sum(self.dx * np.sum(self.mt[None, :, None] * f, axis=(0, 1))))

    def run_to_residual(self, tol: float, max_steps: int, check_every: int = 1):
        while self.steps < max_steps:
            self.step(check_every)
            if self.last_residual < tol:
                return True
        return False

    def set_profiles(self, n, uy, T):
        """f = projected local equilibrium with u_x = 0 (warm start)."""
        n = np.asarray(n, dtype=np.float64)
        self.f = self.equilibrium(n, np.zeros_like(n), np.asarray(uy, dtype=np.float64), np.asarray(T, dtype=np.float64))
