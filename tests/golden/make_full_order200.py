"""Writes full_order200_moments.json: the oracle's moments after 20 RK3 steps of a Fourier
channel with the full-range x rule of order 200 (App. A), for tests/test_gpu_full_order200.py.
Calls only the oracle (its order-200 rule takes ~80 s to build in decimal arithmetic, which is
why the values are stored).  Run from the repository root:
    python tests/golden/make_full_order200.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fdlb as ofd  # noqa: E402

CFG = dict(nx=24, qx_half=100, qy=0, qz=0, kn=0.5, eta0=0.05, T_left=0.95, T_right=1.05, x_quadrature="full")
STEPS = 20


def main():
    o = ofd.Oracle(ofd.Params(**CFG))
    o.step(STEPS)
    M = o.moments()
    out = {"source": "oracle/ (fdlb.Oracle), App. A full-range x rule of order 200", "config": CFG, "steps": STEPS,
           "dt": float(o.dt), "moments": {k: [float(v) for v in M[k]] for k in ("n", "ux", "uy", "T", "qx", "qy", "Pxx", "Pxy")}}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_order200_moments.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
