"""Shared helpers of the GPU parity tests (GPU path vs the FP64 oracle on identical inputs)."""
import os

import numpy as np

from oracle import fdlb as ofd


def lib():
    from paper_2308_15407_gb300 import fdlb
    if not os.path.exists(fdlb.LIB_PATH):
        from paper_2308_15407_gb300 import build
        build.build()
    return fdlb


def oracle_for(p):
    """Oracle instance with the same parameters as a binding Params."""
    return ofd.Oracle(ofd.Params(nx=p.nx, qx_half=p.qx_half, qy=p.qy, qz=p.qz, kn=p.kn, eta0=p.eta0,
                                 T_left=p.T_left, T_right=p.T_right, U_left=p.U_left, U_right=p.U_right,
                                 accel_y=p.accel_y, grid=p.grid, stretch=p.stretch, cfl=p.cfl, dt=p.dt,
                                 j1_shear=p.j1_shear, T_init=p.T_init, chi_model=p.chi_model,
                                 x_quadrature=p.x_quadrature))


def compare(Mg, Mo, rel=1e-12, what=""):
    """Element-wise parity of GPU and oracle moments: relative on n and T, absolute (scaled by
    the profile's own magnitude, at least 1) on u, q and Pi."""
    errs = {}
    for k in ("n", "T"):
        errs[k] = np.max(np.abs(Mg[k] - Mo[k]) / np.abs(Mo[k]))
    for k in ("ux", "uy", "qx", "qy", "Pxx", "Pxy"):
        scale = max(1.0, np.max(np.abs(Mo[k])))
        errs[k] = np.max(np.abs(Mg[k] - Mo[k])) / scale
    tol = dict(n=rel, T=rel, ux=rel, uy=rel, qx=50 * rel, qy=50 * rel, Pxx=10 * rel, Pxy=10 * rel)
    bad = {k: v for k, v in errs.items() if not v <= tol[k]}
    assert not bad, f"{what}: parity failure {bad} (all: {errs})"
    return errs
