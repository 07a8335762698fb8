"""Host-side logic of the learned warm start (no GPU): the node grid agrees with the oracle's,
the feature encoding of the channel parameters, and the mapping of network outputs to
profiles (unit channel mass, no y motion in the 1D reduced form, positive n and T)."""
import math

import numpy as np
import pytest

from oracle import fdlb as ofd
from paper_2308_15407_gb300 import fdlb as F
from paper_2308_15407_gb300 import warmstart as W


@pytest.mark.parametrize("grid", ["uniform", "tanh"])
def test_node_grid_matches_oracle(grid):
    p = F.Params(nx=37, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.1, grid=grid, stretch=1.5)
    x, dx = W.node_grid(p)
    o = ofd.Oracle(ofd.Params(nx=37, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.1, grid=grid, stretch=1.5))
    np.testing.assert_allclose(x, o.x, rtol=0, atol=1e-15)
    np.testing.assert_allclose(dx, o.dx, rtol=1e-14)
    # dx_i = x'(s_i) ds, the scheme's cell width: exactly 1 in total on the uniform grid,
    # 1 + O(ds^2) on the stretched one
    assert abs(dx.sum() - 1.0) < (1e-13 if grid == "uniform" else 1e-3)


def test_features_encoding():
    p = F.Params(nx=20, qx_half=4, qy=4, qz=0, kn=0.05, eta0=0.3, U_left=-0.4, U_right=0.4, accel_y=0.0,
                 flow=F.COUETTE, grid="tanh")
    X = W.features(p)
    assert X.shape == (20, W.NIN) and X.dtype == np.float32
    np.testing.assert_array_equal(X[:, :3], np.tile([0.0, 1.0, 0.0], (20, 1)))
    np.testing.assert_allclose(X[:, 3], math.log10(0.05) + 1.0, rtol=1e-6)
    np.testing.assert_allclose(X[:, 4], 0.5, rtol=1e-6)                  # (0.3 - 0.2)/0.2
    np.testing.assert_allclose(X[:, 5], 0.0)                             # equal wall temperatures
    np.testing.assert_allclose(X[:, 6], 0.6, rtol=1e-6)                  # 0.4/0.25 - 1
    np.testing.assert_allclose(X[:, 7], -1.0)                            # no force
    np.testing.assert_allclose(X[:, 8], 2.0 * W.node_grid(p)[0], rtol=1e-6)
    assert np.all(X[:, 9:] == 0.0)


def test_profiles_from_outputs():
    p2 = F.Params(nx=30, qx_half=4, qy=4, qz=0, kn=0.1, eta0=0.1, U_left=-0.3, U_right=0.3, grid="tanh")
    x, dx = W.node_grid(p2)
    M = {"n": 1.0 + 0.02 * x ** 2, "uy": 0.3 * x, "T": 1.0 + 0.01 * np.cos(x)}
    n, uy, T = W.profiles(W.targets(M), p2)
    assert abs(np.sum(dx * n) - 1.0) < 1e-13                            # unit channel mass
    np.testing.assert_allclose(n / n[0], M["n"] / M["n"][0], rtol=1e-6)   # shape kept (float32 round trip)
    np.testing.assert_allclose(uy, M["uy"], atol=1e-7)
    np.testing.assert_allclose(T, M["T"], rtol=1e-7)
    # 1D reduced form: no y velocity; floors keep n, T positive
    p1 = F.Params(nx=30, qx_half=4, qy=0, qz=0, kn=0.1, eta0=0.1)
    bad = np.tile(np.array([[-50.0, 3.0, -50.0]], dtype=np.float32), (30, 1))
    n, uy, T = W.profiles(bad, p1)
    assert np.all(uy == 0.0) and np.all(T >= 0.2) and np.all(n > 0)
    assert abs(np.sum(W.node_grid(p1)[1] * n) - 1.0) < 1e-13
