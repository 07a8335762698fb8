"""Full-range x quadrature at App. A's order 200 (qx_half = 100, 200 x-velocities) against the
oracle: FP64 1e-12 and FP32 1e-5 after 20 steps of a Fourier channel, both precisions in one
batch.  The closure's x projection runs in blocks of 16 of the 200 orthonormal polynomials on
the 102-point Gauss-Hermite auxiliary rule.  The oracle's moments are stored in
tests/golden/full_order200_moments.json, written by tests/golden/make_full_order200.py from
oracle/ alone (its order-200 rule takes ~80 s to build in decimal arithmetic)."""
import json
import os

import numpy as np
import pytest

from gpu_common import compare, lib

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_order200_moments.json")


def test_full_range_order_200_matches_oracle():
    ref = json.load(open(GOLDEN))
    F = lib()
    cfg = ref["config"]
    s = F.Solver([F.Params(**cfg, precision="fp64"), F.Params(**cfg, precision="fp32")])
    s.set_schedule("tiled")
    s.step(ref["steps"])
    assert abs(s.dt[0] - ref["dt"]) <= 1e-14 * ref["dt"]
    Mo = {k: np.asarray(v) for k, v in ref["moments"].items()}
    compare(s.moments(0), Mo, 1e-12, "order 200, fp64")
    compare(s.moments(1), Mo, 1e-5, "order 200, fp32")
