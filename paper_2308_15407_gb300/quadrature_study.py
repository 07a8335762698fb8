"""Velocity-quadrature studies of Sec. IV and App. A in the paper's geometry.

  python -m paper_2308_15407_gb300.quadrature_study [table1|fullhalf|heatflux|mfr|mfr_kn] [--cells-per-sigma 20]

table1    The convergence test behind the paper's Table 1: for each flow (Fourier with
          Delta T = 0.1, Couette with U_w = 1, Poiseuille with a_y = 0.001 in v^2/sigma),
          confinement R in {4, 10} and reduced density eta0 in {0.01, 0.1, 0.2}, the error
          eps = max |M - M_ref| / (max M_ref - min M_ref) (M = T, u_y, u_y) of half-range orders
          4 .. 29 per side against a reference, and the smallest order with eps < 1 %.  The
          paper's reference is order 200 and its spacing sigma/100; here the reference is
          32 per side, and the spacing is an argument.  --flows / --etas select a subset,
          --steady profile stops on the change of the profiles instead of the residual.
fullhalf  App. A's comparison (R = 10, eta0 = 0.01): full-range orders 16 .. 200 against the
          same reference, beside half-range orders.
heatflux  Fourier flow (Delta T = 0.1): the heat flux q_x / n0 across the channel against the
          Knudsen number (varied through R at fixed eta0) for eta0 in {0.01, 0.1, 0.2}.
mfr       The Poiseuille mass flow rate against Kn for the half-range orders 8, 16, 32, 64, and
          100 above Kn = 1 (the orders of Sec. IV's mass-flow figure), R = 10, a_y = 0.001.
mfr_kn    The mass flow rate against Kn for R in {2, 5, 10, 20} as Sec. IV computes it: order 8
          up to Kn = 1, order 100 above (Kn = 2 and 5 here, with order 8 beside them).

Steady states: table1, fullhalf and heatflux in FP64 to per-step residual 1e-9 under a
wall-clock cap (table1 optionally by the change of its profiles); mfr and mfr_kn in FP32 by the
change of the mass flow over a time unit (the per-step residual stops those flows early, since
dt shrinks with the largest velocity of the order).  RET-FM contact value (the paper's); Q_y =
5 for table1's 2D flows, 4 for the mass-flow runs.  Everything runs through the public binding;
the output is one JSON document.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

FLOWS = [("fourier", dict(dT=0.1), "T"), ("couette", dict(U_w=1.0), "uy"), ("poiseuille", dict(a_y=0.001), "uy")]
HALF_ORDERS = (4, 6, 8, 11, 15, 20, 24, 29)
REF_ORDER = 32
TOL = 1e-9


def _steady(F, dicts, cap_s):
    import torch
    s = F.Solver([F.Params(**d) for d in dicts])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        s.run(TOL, 5_000_000, check_every=2000, timeout_s=cap_s)
    except F.FdlbError:
        pass
    torch.cuda.synchronize()
    return s, time.perf_counter() - t0


def _eps(M, R):
    return float(np.max(np.abs(M - R)) / (R.max() - R.min()))


def table1(cells_per_sigma=20, cap_s=900.0, flows=None, steady="residual", precision="fp64", window=1.0, rel=1e-5,
           etas=(0.01, 0.1, 0.2)):
    """steady = "residual": each instance frozen at per-step residual TOL; "profile": the batch
    stepped until every instance's monitored profile M changed by less than rel x (its range)
    over a time unit (reading R20: at small dt the per-step residual stops a Poiseuille flow
    early)."""
    from . import fdlb as F
    from . import workloads as W
    cases, dicts = [], []
    for fl, kw, key in FLOWS:
        if flows and fl not in flows:
            continue
        for R in (4, 10):
            for eta in etas:
                for q in (REF_ORDER,) + HALF_ORDERS:
                    dicts.append(W.paper_geometry(R, eta, qx_half=q, cells_per_sigma=cells_per_sigma, flow=fl,
                                                  precision=precision, **kw))
                cases.append((fl, key, R, eta))
    if steady == "profile":
        s = F.Solver([F.Params(**d) for d in dicts])
        keys = [c[1] for c in cases for _ in range(1 + len(HALF_ORDERS))]

        def mon(i):
            M = s.moments(i)[keys[i]]
            return M, float(M.max() - M.min())
        _, change, nsteps, sec, _, _ = _step_until_steady(F, s, len(dicts), mon, cap_s, window, rel)
        done = change < rel
        st = np.where(done, F.CONVERGED, F.ACTIVE)
        steps = np.full(len(dicts), nsteps)
        crit = f"profile change < {rel} x range over >= {window} time units"
    else:
        s, sec = _steady(F, dicts, cap_s)
        _, st, steps = s.status()
        crit = f"per-step residual < {TOL}"
    out = {"cells_per_sigma": cells_per_sigma, "reference_order": REF_ORDER, "seconds": sec, "criterion": crit,
           "precision": precision, "all_converged": bool(np.all(st == F.CONVERGED)), "cases": []}
    n = 1 + len(HALF_ORDERS)
    for c, (fl, key, R, eta) in enumerate(cases):
        base = c * n
        ref = s.moments(base)[key]
        eps = {q: _eps(s.moments(base + 1 + j)[key], ref) for j, q in enumerate(HALF_ORDERS)}
        conv = [bool(st[base + j] == F.CONVERGED) for j in range(n)]
        first = next((q for q in HALF_ORDERS if eps[q] < 0.01), None)
        out["cases"].append({"flow": fl, "R": R, "eta0": eta, "eps": eps, "smallest_order_below_1pct": first,
                             "converged": all(conv), "steps_reference": int(steps[base])})
    return out


def fullhalf(cells_per_sigma=20, cap_s=900.0, full_orders=(16, 32, 64, 100, 200), half_orders=(8, 16, 29)):
    from . import fdlb as F
    from . import workloads as W
    dicts = []
    for fl, kw, key in FLOWS:
        dicts.append(W.paper_geometry(10, 0.01, qx_half=REF_ORDER, cells_per_sigma=cells_per_sigma, flow=fl, **kw))
        for q in half_orders:
            dicts.append(W.paper_geometry(10, 0.01, qx_half=q, cells_per_sigma=cells_per_sigma, flow=fl, **kw))
        for o in full_orders:
            dicts.append(W.paper_geometry(10, 0.01, qx_half=o // 2, cells_per_sigma=cells_per_sigma, flow=fl,
                                          x_quadrature="full", **kw))
    s, sec = _steady(F, dicts, cap_s)
    _, st, steps = s.status()
    n = 1 + len(half_orders) + len(full_orders)
    out = {"cells_per_sigma": cells_per_sigma, "reference": f"half-range {REF_ORDER} per side", "seconds": sec,
           "all_converged": bool(np.all(st == F.CONVERGED)), "flows": []}
    for fi, (fl, _, key) in enumerate(FLOWS):
        base = fi * n
        ref = s.moments(base)[key]
        half = {q: _eps(s.moments(base + 1 + j)[key], ref) for j, q in enumerate(half_orders)}
        full = {o: _eps(s.moments(base + 1 + len(half_orders) + j)[key], ref) for j, o in enumerate(full_orders)}
        row = {"flow": fl, "half_eps": half, "full_eps": full,
               "converged": [bool(x == F.CONVERGED) for x in st[base:base + n]]}
        if fl == "poiseuille":
            mfr = lambda i: float(np.mean(s.moments(i)["n"] * s.moments(i)["uy"]))
            row["mean_n_uy"] = {"reference": mfr(base),
                                "full": {o: mfr(base + 1 + len(half_orders) + j) for j, o in enumerate(full_orders)}}
        out["flows"].append(row)
    return out


def heatflux(cells_per_sigma=20, cap_s=600.0, R_values=(2, 3, 4, 6, 10, 20), qx_half=11):
    from . import fdlb as F
    from . import workloads as W
    dicts, tags = [], []
    for eta in (0.01, 0.1, 0.2):
        for R in R_values:
            d = W.paper_geometry(R, eta, qx_half=qx_half, cells_per_sigma=max(cells_per_sigma, int(np.ceil(60 / (R - 1)))),
                                 flow="fourier", dT=0.1)
            dicts.append(d)
            chi0 = (2.0 - eta) / (2.0 * (1.0 - eta) ** 3)
            tags.append({"eta0": eta, "R": R, "Kn_L": 1.0 / (6.0 * np.sqrt(2.0) * eta * chi0 * R)})
    s, sec = _steady(F, dicts, cap_s)
    _, st, _ = s.status()
    rows = []
    for i, t in enumerate(tags):
        M = s.moments(i)
        # q_x is uniform at steady state (up to truncation); report its channel mean and spread.
        # Channel-width units: q_x in n0 (k_B T0/m)^(3/2), the paper's q_x / n0.
        rows.append({**t, "qx_over_n0": float(np.mean(M["qx"])), "qx_spread": float(np.ptp(M["qx"])),
                     "converged": bool(st[i] == F.CONVERGED)})
    return {"cells_per_sigma": cells_per_sigma, "qx_half": qx_half, "seconds": sec, "rows": rows}


def mfr(cells_per_sigma=20, cap_s=600.0, R=10, kn_values=(0.1, 0.5, 1.0, 2.0, 5.0), orders=(8, 16, 32, 64),
        q_large=100, window=1.0, rel=2e-5):
    """G = mean of n u_y over the channel / a_y (channel-width units), the paper's m-dot/m-dot_0
    (Sec. IV), for each (Kn, order).  FP32 storage.  Each instance's dt follows its largest
    velocity (~22 thermal speeds at order 100), so a per-step residual is no common measure of
    convergence; instead the batch is stepped in chunks covering at least `window` time units
    of the smallest dt, and an instance counts as steady once G changed by less than `rel`
    (relative) over its last chunk.  Stops when all are steady or at the wall-clock cap."""
    from . import fdlb as F
    from . import workloads as W
    dicts, tags = [], []
    for kn in kn_values:
        eta0 = W.eta_for_knudsen(float(kn), R)
        cps = max(cells_per_sigma, int(np.ceil(60 / (R - 1.0))))
        for q in tuple(orders) + ((q_large,) if kn > 1.0 else ()):
            dicts.append(W.paper_geometry(R, eta0, qx_half=q, cells_per_sigma=cps, precision="fp32",
                                          flow="poiseuille", a_y=0.001, qy=4))
            tags.append({"Kn_L": float(kn), "eta0": float(eta0), "qx_half": q})
    out = _mfr_steady(F, dicts, tags, cap_s, window, rel)
    out.update(R=R, cells_per_sigma=cells_per_sigma)
    return out


def _step_until_steady(F, s, n, monitor, cap_s, window, rel):
    """Steps batch s in chunks of at least `window` time units of its smallest dt until, for
    every instance i, monitor(i) = (values, scale) changed by less than rel * scale (largest
    element) over the last chunk, or an instance failed, or the wall-clock cap.  Returns
    (last values, last relative changes, steps, seconds, dt, steps per chunk).  The monitor's
    reads of the moments synchronise with the device, so the clock is right at chunk ends."""
    dt = np.asarray(s.dt, dtype=float)
    chunk = int(np.ceil(window / dt.min()))
    prev = [None] * n
    change = np.full(n, np.inf)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < cap_s:
        s.step(chunk)
        steps += chunk
        for i in range(n):
            v, scale = monitor(i)
            change[i] = np.inf if prev[i] is None else float(np.max(np.abs(v - prev[i]))) / scale
            prev[i] = v
        failed = s.status()[1] != F.ACTIVE
        if np.all((change < rel) | failed):
            break
    return prev, change, steps, time.perf_counter() - t0, dt, chunk


def _mfr_steady(F, dicts, tags, cap_s, window, rel):
    """Steps the Poiseuille batch until G = mean(n u_y)/a_y of every instance changed by less
    than `rel` (relative) over a chunk of at least `window` time units (or the cap); one row
    per instance."""
    s = F.Solver([F.Params(**d) for d in dicts])

    def G(i):
        g = float(np.mean(s.moments(i)["n"] * s.moments(i)["uy"])) / dicts[i]["accel_y"]
        return np.array([g]), abs(g)
    vals, change, steps, sec, dt, chunk = _step_until_steady(F, s, len(dicts), G, cap_s, window, rel)
    prev = np.array([v[0] for v in vals])
    _, st, _ = s.status()
    rows = [{**t, "G": float(prev[i]), "last_change": float(change[i]), "time_units": float(steps * dt[i]),
             "steady": bool(change[i] < rel), "status": int(st[i])} for i, t in enumerate(tags)]
    return {"steps": steps, "chunk": chunk, "seconds": sec,
            "criterion": f"relative change of G < {rel} over a chunk of >= {window} time units", "rows": rows}


def mfr_kn(cells_per_sigma=20, cap_s=720.0, R_values=(2, 5, 10, 20), points=8, kn_large=(2.0, 5.0), q_small=8,
           q_large=100, R_large=(2, 5, 10), window=1.0, rel=2e-5):
    """Sec. IV's mass-flow figure: for each R, the Knudsen numbers of workloads.knudsen_sweep (from
    the smallest reachable with eta0 <= 0.2 to 1) at order q_small, and for R in R_large the
    Knudsen numbers kn_large at order q_large (the paper's switch above Kn = 1) and at q_small
    (R = 20 at order 100 would need ~5e5 steps of dt ~6e-5 on its 380 nodes); convergence as in
    mfr()."""
    from . import fdlb as F
    from . import workloads as W
    base, btags = W.knudsen_sweep(R_values=R_values, points=points, kn_max=1.0, qx_half=q_small,
                                  cells_per_sigma=cells_per_sigma)
    dicts = list(base)
    tags = [{"R": R, "Kn_L": kn, "eta0": eta, "qx_half": q_small} for (R, kn, eta) in btags]
    for R in R_large:
        cps = max(cells_per_sigma, int(np.ceil(60 / (R - 1.0))))
        for kn in kn_large:
            eta0 = W.eta_for_knudsen(float(kn), R)
            for q in (q_small, q_large):
                dicts.append(W.paper_geometry(R, eta0, qx_half=q, cells_per_sigma=cps, precision="fp32",
                                              flow="poiseuille", a_y=0.001, qy=4))
                tags.append({"R": R, "Kn_L": float(kn), "eta0": float(eta0), "qx_half": q})
    out = _mfr_steady(F, dicts, tags, cap_s, window, rel)
    out.update(cells_per_sigma=cells_per_sigma)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["table1", "fullhalf", "heatflux", "mfr", "mfr_kn"])
    ap.add_argument("--cells-per-sigma", type=int, default=20)
    ap.add_argument("--cap-s", type=float, default=900.0)
    ap.add_argument("--flows", default=None, help="table1: comma-separated subset of fourier,couette,poiseuille")
    ap.add_argument("--steady", default="residual", choices=["residual", "profile"], help="table1's stopping rule")
    ap.add_argument("--precision", default="fp64", help="table1's storage precision")
    ap.add_argument("--etas", default="0.01,0.1,0.2", help="table1's reduced densities")
    a = ap.parse_args()
    if a.what == "table1":
        out = table1(a.cells_per_sigma, a.cap_s, flows=a.flows.split(",") if a.flows else None, steady=a.steady,
                     precision=a.precision, etas=tuple(float(e) for e in a.etas.split(",")))
    else:
        fn = {"fullhalf": fullhalf, "heatflux": heatflux, "mfr": mfr, "mfr_kn": mfr_kn}[a.what]
        out = fn(a.cells_per_sigma, a.cap_s)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
