"""The paper's confinement (R = L/sigma = 4) for a dense gas at rest (Sec. IV, density next to
a wall): with the Fischer-Methfessel contact value the steady density rises at the walls
(layering) while the total normal stress stays uniform; with chi_SET the uniform rest state
is already steady."""
import numpy as np
import pytest

from gpu_common import lib, oracle_for
from oracle import fdlb as ofd
from paper_2308_15407_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_density_layering_at_rest():
    F = lib()
    d = workloads.paper_geometry(4, 0.1)
    s = F.Solver([F.Params(**d), F.Params(**{**d, "chi_model": "set"})])
    rc = s.run(1e-10, 300000, check_every=2000)
    r, st, ns = s.status()
    assert rc == 0 and st.tolist() == [F.CONVERGED, F.CONVERGED], (r, st, ns)
    n_fm, n_set = s.moments(0)["n"], s.moments(1)["n"]
    dx = 1.0 / d["nx"]
    # mass is conserved (mean density 1)
    assert abs(np.sum(n_fm) * dx - 1.0) < 1e-10 and abs(np.sum(n_set) * dx - 1.0) < 1e-10
    # SET: the uniform rest state stays uniform; RET-FM: contact density above the bulk
    assert np.max(np.abs(n_set - 1.0)) < 1e-9
    mid = n_fm[d["nx"] // 2]
    assert n_fm[0] > 1.02 * mid and n_fm[-1] > 1.02 * mid     # measured 1.033
    assert abs(n_fm[0] / n_fm[-1] - 1.0) < 1e-8              # mirror symmetry
    M = s.moments(0)
    # the gas stays at rest up to truncation: the wall node carries a ~1e-5 discretisation
    # velocity next to the steep density layer, the interior ~1e-8
    assert np.max(np.abs(M["ux"])) < 1e-4 and np.max(np.abs(M["ux"][10:-10])) < 1e-6
    # momentum balance at rest: kinetic plus collisional normal stress, Pi_xx + b rho^2 chi T
    # with chi of the averaged density, is uniform across the channel (truncation only)
    o = oracle_for(F.Params(**d))
    P = M["Pxx"] + 4.0 * d["eta0"] * M["n"] ** 2 * ofd.chi_set(d["eta0"] * (o.Wfm @ M["n"])) * M["T"]
    assert (P.max() - P.min()) / P.mean() < 1e-4
