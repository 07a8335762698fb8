"""Steady-state conservation in the channel (closed-form invariants of the steady 1D kinetic
equation): Fourier q_x uniform; Pi_xx + b rho^2 chi T uniform (all flows); Couette Pi_xy
uniform.  The discrete steady states satisfy them to truncation: the spreads must shrink
under grid refinement (the measured rate is first order, set by the wall closure)."""
import numpy as np
import pytest

from gpu_common import lib
from oracle import fdlb as ofd

pytestmark = pytest.mark.gpu

FOURIER = dict(qx_half=6, qy=0, qz=0, kn=0.1, eta0=0.1, T_left=0.95, T_right=1.05)
COUETTE = dict(qx_half=6, qy=6, qz=0, kn=0.1, eta0=0.1, U_left=-0.3, U_right=0.3)
NS = (50, 100)


def spread(v):
    return (v.max() - v.min()) / np.mean(np.abs(v))


def test_conserved_fluxes_uniform_and_converging():
    F = lib()
    cases = [("fourier", N, FOURIER) for N in NS] + [("couette", N, COUETTE) for N in NS]
    s = F.Solver([F.Params(nx=N, **d) for _, N, d in cases])
    rc = s.run(1e-11, 200000, check_every=2000)
    r, st, ns = s.status()
    assert rc == 0 and all(x == F.CONVERGED for x in st), (r, st, ns)
    sp = {}
    for i, (name, N, d) in enumerate(cases):
        M = s.moments(i)
        eta0 = d["eta0"]
        P = M["Pxx"] + 4.0 * eta0 * M["n"] ** 2 * ofd.chi_set(eta0 * M["n"]) * M["T"]
        sp[(name, N, "P")] = spread(P)
        sp[(name, N, "flux")] = spread(M["qx"] if name == "fourier" else M["Pxy"])
    for name in ("fourier", "couette"):
        for q in ("P", "flux"):
            coarse, fine = sp[(name, NS[0], q)], sp[(name, NS[1], q)]
            assert fine < 5e-3, (name, q, fine)
            assert fine < 0.6 * coarse, (name, q, coarse, fine)
