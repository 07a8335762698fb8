"""Seeded synthetic workloads (parameter sets only; no arithmetic of the method).

Used by the tests and the benchmark to build identical inputs for the CUDA path and for the
oracle.  Each function returns a list of plain dicts with the keys of ``fdlb.Params``
(``knudsen_sweep`` also returns the confinement ratio and Knudsen number of each).
"""
import numpy as np

FOURIER, COUETTE, POISEUILLE = 0, 1, 2


def couette_sweep(precision="fp32"):
    """Couette flow: Nx = 200 tanh-stretched (A = 1.5), walls at T = 1 moving at -0.42/+0.42,
    eta0 in {0.1, 0.2, 0.3, 0.4} x Kn in {0.05, 0.1, 0.5}, 6 half-range per side x 6 x 4."""
    return [dict(nx=200, qx_half=6, qy=6, qz=4, kn=kn, eta0=eta, U_left=-0.42, U_right=0.42, grid="tanh",
                 stretch=1.5, flow=COUETTE, precision=precision)
            for eta in (0.1, 0.2, 0.3, 0.4) for kn in (0.05, 0.1, 0.5)]


def fourier_5000():
    """Fourier flow, Nx = 50 uniform, walls 0.95/1.05, eta0 = 0.1, Kn = 0.1, 4 x 4 x 4 per side."""
    return [dict(nx=50, qx_half=4, qy=4, qz=4, kn=0.1, eta0=0.1, T_left=0.95, T_right=1.05, flow=FOURIER)]


def batched_sweep(count=2048, seed=23084, precision="fp32"):
    """Parameter sweep of mixed flows in one batch.  Draws, in this order per instance, from
    numpy's PCG64(seed): flow uniform in {Fourier, Couette, Poiseuille}; Nx uniform integer in
    [32, 512]; half-range order per side in {4, 6, 8}; log10 Kn uniform in [-2, 0]; eta0 uniform
    in [0.01, 0.45]; Delta T uniform in [0, 0.2]; wall speed uniform in [0, 0.5]; force uniform in
    [0, 0.1].  Every draw is made for every instance (a fixed stream); each flow uses only its
    own parameter (Fourier: walls 1 -+ Delta T; Couette: walls at T = 1 moving -+ U; Poiseuille:
    walls at rest, a_y).  Fourier instances use the 1D reduced velocity set (q_y = q_z = 0),
    Couette and Poiseuille the 2D reduced set with q_y = 4; uniform grids."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        flow = int(rng.integers(0, 3))
        nx = int(rng.integers(32, 513))
        q = int(rng.choice([4, 6, 8]))
        kn = float(10.0 ** rng.uniform(-2.0, 0.0))
        eta = float(rng.uniform(0.01, 0.45))
        dT = float(rng.uniform(0.0, 0.2))
        uw = float(rng.uniform(0.0, 0.5))
        ay = float(rng.uniform(0.0, 0.1))
        p = dict(nx=nx, qx_half=q, kn=kn, eta0=eta, flow=flow, precision=precision, grid="uniform")
        if flow == FOURIER:
            p.update(qy=0, qz=0, T_left=1.0 - dT, T_right=1.0 + dT)
        elif flow == COUETTE:
            p.update(qy=4, qz=0, U_left=-uw, U_right=uw)
        else:
            p.update(qy=4, qz=0, accel_y=ay)
        out.append(p)
    return out


def couette_family(count, seed, nx=200, qx_half=6, qy=6, qz=4, grid="tanh", precision="fp32",
                   eta=(0.05, 0.25), log10_kn=(-1.5, -0.3), wall=(0.3, 0.5)):
    """Couette instances with eta0, log10 Kn and wall speed U (walls at -U/+U, T = 1) drawn
    uniformly from the given ranges by PCG64(seed), in that order per instance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        e = float(rng.uniform(*eta))
        kn = float(10.0 ** rng.uniform(*log10_kn))
        u = float(rng.uniform(*wall))
        out.append(dict(nx=nx, qx_half=qx_half, qy=qy, qz=qz, kn=kn, eta0=e, U_left=-u, U_right=u, grid=grid,
                        stretch=1.5, flow=COUETTE, precision=precision))
    return out


def paper_geometry(R, eta0, qx_half=8, T_w=1.0, cells_per_sigma=100, precision="fp64", flow="rest", dT=0.0,
                   U_w=0.0, a_y=0.0, qy=5, x_quadrature="half"):
    """The paper's own confinement (Sec. IV): walls L = R sigma apart whose molecule centres
    reach +-(L - sigma)/2, so the computational width is D = (R - 1) sigma, i.e.
    sigma = D/(R - 1) in channel-width units; the Kn of Sec. II A, referred to D, is
    1/(6 sqrt(2) eta0 chi(eta0) (R - 1)), and Delta x = sigma/cells_per_sigma (100 in the
    paper).  The Fischer-Methfessel contact value (Eq. chi_ret) gives the density layering
    next to the walls.

    flow: "rest" (1D reduced, walls at T_w), "fourier" (1D reduced, walls at T_w -+ dT),
    "couette" (2D reduced with qy, walls at -+U_w and T_w), "poiseuille" (2D reduced, walls at
    rest, acceleration a_y).  The paper measures lengths in sigma (its L_c = R - 1) and speeds
    in sqrt(k_B T_w/m); a_y is given in those units, v^2/sigma, and converted to the
    channel-width units used here, a_y (R - 1).  x_quadrature: "half" (Sec. III A 2) or
    "full" (order 2 qx_half, App. A)."""
    chi0 = (2.0 - eta0) / (2.0 * (1.0 - eta0) ** 3)
    kn = 1.0 / (6.0 * np.sqrt(2.0) * eta0 * chi0 * (R - 1.0))
    d = dict(nx=int(round(cells_per_sigma * (R - 1))), qx_half=qx_half, qy=0, qz=0, kn=float(kn), eta0=eta0,
             T_left=T_w, T_right=T_w, chi_model="ret-fm", precision=precision, flow=0, x_quadrature=x_quadrature)
    if flow == "rest":
        return d
    if flow == "fourier":
        d.update(T_left=T_w - dT, T_right=T_w + dT)
    elif flow == "couette":
        d.update(qy=qy, U_left=-U_w, U_right=U_w, flow=1)
    elif flow == "poiseuille":
        d.update(qy=qy, accel_y=float(a_y * (R - 1.0)), flow=2)
    else:
        raise ValueError("flow must be rest, fourier, couette or poiseuille")
    return d


def eta_for_knudsen(kn_L, R, eta_hi=0.49):
    """eta0 with 1/(6 sqrt(2) eta0 chi(eta0) R) = kn_L (the Kn of Sec. II A referred to
    L = R sigma), by bisection on the increasing eta0 chi(eta0); None when kn_L needs
    eta0 >= eta_hi."""
    target = 1.0 / (6.0 * np.sqrt(2.0) * kn_L * R)
    g = lambda e: e * (2.0 - e) / (2.0 * (1.0 - e) ** 3)
    if g(eta_hi) < target:
        return None
    lo, hi = 0.0, eta_hi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def knudsen_sweep(R_values=(2, 5, 10, 20), points=8, kn_max=1.0, eta_max=0.2, a_y=0.001, qx_half=8, qy=4,
                  cells_per_sigma=20, min_cells=60, precision="fp32"):
    """Poiseuille mass-flow sweep of Sec. IV (mass flow rate against Kn for several R) in the
    paper's geometry: for each R, `points` Knudsen numbers (referred to L = R sigma) spaced
    logarithmically from the smallest one reachable with eta0 <= eta_max (higher densities
    are linearly unstable with these velocity sets) to kn_max; eta0 from eta_for_knudsen;
    acceleration a_y in v^2/sigma; Delta x = sigma/cells_per_sigma, at least min_cells cells.
    Returns (dicts, tags) with tags[i] = (R, Kn_L, eta0)."""
    dicts, tags = [], []
    for R in R_values:
        g_max = eta_max * (2.0 - eta_max) / (2.0 * (1.0 - eta_max) ** 3)
        kn_min = 1.0 / (6.0 * np.sqrt(2.0) * g_max * R)
        for kn in np.geomspace(kn_min * 1.0001, kn_max, points):
            eta0 = eta_for_knudsen(float(kn), R)
            cps = max(cells_per_sigma, int(np.ceil(min_cells / (R - 1.0))))
            d = paper_geometry(R, eta0, qx_half=qx_half, cells_per_sigma=cps, precision=precision,
                               flow="poiseuille", a_y=a_y, qy=qy)
            dicts.append(d)
            tags.append((R, float(kn), float(eta0)))
    return dicts, tags

