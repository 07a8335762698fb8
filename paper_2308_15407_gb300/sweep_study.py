"""Steady-state study of the seeded parameter sweep and the learned warm start.

  python -m paper_2308_15407_gb300.sweep_study [--instances 2048] [--test 512] [--cap-s 240]
  python -m paper_2308_15407_gb300.sweep_study --configs      # the named set-ups C1-C3

Sweep (the mixed batch of ``workloads.batched_sweep``: flow, Nx in [32, 512], Q_x^h in
{4, 6, 8}, Kn log-uniform in [0.01, 1], eta0 in [0.01, 0.45], wall and force parameters,
seed 23084): one batch solved to per-step residual 1e-8 with per-instance freezing, under a
wall-clock cap (the slowest instances, small Kn on fine grids, need ~10^5 RK3 steps).
Reported: instances converged / failed / still active at the cap, solves/s, the RK3 steps of
the converged instances, and the schedule the autotuner picked.

Warm start: the network (``warmstart.WarmStart``) is trained on the steady states of the
sweep's converged instances, then a fresh seeded batch drawn from the same distribution
(seed 230855) is solved twice, from the uniform state and from the network's profiles.
Reported: steps and wall time of both, their solves/s, and the plain FP64 per-instance GPU
rate on a sample of the converged instances (each solved alone in FP64 storage), which
gives the ratio batched + warm FP32 solves/s over plain FP64 per-instance solves/s.

Everything runs through the library's public binding; the output is one JSON document.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

TOL = 1e-8


def _solve(s, F, cap_s, check=2000, max_steps=2_000_000):
    """fdlb_run to TOL under a wall-clock cap; returns (seconds, return code)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        rc = s.run(TOL, max_steps, check_every=check, timeout_s=cap_s)
    except F.FdlbError as e:
        rc = e.code
    torch.cuda.synchronize()
    return time.perf_counter() - t0, rc


def _summary(s, F, seconds):
    _, st, steps = s.status()
    conv = st == F.CONVERGED
    q = lambda a, p: float(np.percentile(a, p)) if len(a) else None
    cs = steps[conv]
    return {"instances": int(s.count), "converged": int(conv.sum()),
            "failed_nonfinite": int((st == F.FAILED_NONFINITE).sum()),
            "failed_unphysical": int((st == F.FAILED_UNPHYSICAL).sum()),
            "still_active": int((st == F.ACTIVE).sum()), "seconds": seconds,
            "solves_per_s": float(conv.sum()) / seconds,
            "steps_converged": {"min": int(cs.min()) if len(cs) else None, "p50": q(cs, 50), "p90": q(cs, 90),
                                "max": int(cs.max()) if len(cs) else None, "sum": int(cs.sum())},
            "node_velocity_updates": float(sum(int(n) * a * b for n, a, b in zip(steps, s.nx, s.nvel)))}


def run(instances=2048, test=512, cap_s=240.0, test_cap_s=120.0, plain_sample=8, train_steps=2000, device="cuda"):
    import torch
    from . import fdlb as F
    from . import workloads
    from .warmstart import WarmStart
    out = {"tolerance": TOL}

    # ---- the sweep
    sweep = [F.Params(**d) for d in workloads.batched_sweep(instances, seed=23084)]
    s = F.Solver(sweep, device=device)
    sec, rc = _solve(s, F, cap_s)
    out["sweep"] = _summary(s, F, sec)
    out["sweep"]["run_return"] = int(rc)
    out["sweep"]["schedule"] = s.schedule()[0]
    out["sweep"]["smem_resident_eligible"] = int(s.schedule_mix().sum())
    out["sweep"]["updates_per_s"] = out["sweep"]["node_velocity_updates"] / sec

    # ---- warm-start network trained on the sweep's steady states
    X, Y = WarmStart.dataset(s)
    s.close()
    t0 = time.perf_counter()
    warm = WarmStart(max_points=X.shape[0], seed=7, device=device)
    hist = warm.fit(X, Y, steps=train_steps)
    torch.cuda.synchronize()
    out["network"] = {"train_instances": out["sweep"]["converged"], "train_points": int(X.shape[0]),
                      "adam_steps": train_steps, "loss_first_last": [hist[0], hist[-1]],
                      "seconds": time.perf_counter() - t0}

    # ---- fresh batch: cold vs warm
    fresh = [F.Params(**d) for d in workloads.batched_sweep(test, seed=230855)]
    sc = F.Solver(fresh, device=device)
    sec_c, rc_c = _solve(sc, F, test_cap_s)
    out["cold"] = _summary(sc, F, sec_c)
    _, st_c, n_c = sc.status()
    sw = F.Solver(fresh, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    warm.apply(sw)
    sec_w, rc_w = _solve(sw, F, test_cap_s)
    sec_w += 0.0
    out["warm"] = _summary(sw, F, time.perf_counter() - t0)
    _, st_w, n_w = sw.status()
    both = (st_c == F.CONVERGED) & (st_w == F.CONVERGED)
    out["warm_vs_cold"] = {"converged_by_both": int(both.sum()),
                           "steps_ratio_median": float(np.median(n_w[both] / n_c[both])) if both.any() else None,
                           "steps_sum_cold_warm": [int(n_c[both].sum()), int(n_w[both].sum())]}
    # profiles of the two solves of the same instances (both at residual TOL)
    errs = []
    for i in np.nonzero(both)[0][:64]:
        Mc, Mw = sc.moments(int(i)), sw.moments(int(i))
        errs.append(max(float(np.max(np.abs(Mw["n"] - Mc["n"]) / Mc["n"])), float(np.max(np.abs(Mw["T"] - Mc["T"]) / Mc["T"]))))
    out["warm_vs_cold"]["n_T_rel_diff_max_first64"] = max(errs) if errs else None

    # ---- plain FP64 per-instance GPU solves on a sample of the converged fresh instances
    conv = [int(i) for i in np.nonzero(st_w == F.CONVERGED)[0]]
    rng = np.random.Generator(np.random.PCG64(5))
    pick = sorted(rng.choice(conv, size=min(plain_sample, len(conv)), replace=False).tolist()) if conv else []
    tot = 0.0
    per = []
    for i in pick:
        p = F.Params(**{**fresh[i].__dict__, "precision": "fp64"})
        s1 = F.Solver([p], device=device)
        sec1, _ = _solve(s1, F, 600.0)
        tot += sec1
        per.append({"instance": i, "seconds": sec1, "steps": int(s1.status()[2][0]),
                    "converged": bool(s1.status()[1][0] == F.CONVERGED)})
        s1.close()
    plain = len(pick) / tot if tot else None
    out["plain_fp64_per_instance"] = {"sample": per, "solves_per_s": plain}
    out["batched_warm_over_plain_fp64"] = out["warm"]["solves_per_s"] / plain if plain else None
    out["batched_cold_over_plain_fp64"] = out["cold"]["solves_per_s"] / plain if plain else None
    sc.close()
    sw.close()
    return out


def _timed_steps(s, n):
    """Seconds of n RK3 steps by CUDA events on the solver's stream, and the node-velocity
    updates they performed."""
    import torch
    n0 = s.status()[2].copy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(n)
    e1.record(s.stream)
    torch.cuda.synchronize()
    done = s.status()[2] - n0
    return e0.elapsed_time(e1) * 1e-3, float(sum(int(d) * a * b for d, a, b in zip(done, s.nx, s.nvel)))


def configs(device="cuda", c2_cap_s=240.0, c3_cap_s=180.0):
    """The named set-ups beside the sweep: C1 Fourier (Nx = 50 uniform, walls 0.95 / 1.05,
    eta0 = 0.1, Kn = 0.1, 4 per side x 4 x 4 = 128 velocities, FP64), 5000 RK3 steps of one
    instance and 500 steps of 2048 replicas; C2 the Couette sweep (12 instances, Nx = 200 tanh,
    12 x 6 x 4 velocities) in FP64 to residual 1e-10 and in FP32 storage to 1e-8, with the FP32
    profiles against the FP64 ones; C3 Poiseuille (a_y = 0.05, Nx = 400 tanh, walls at rest,
    eta0 in {0.05, 0.2, 0.35} x Kn = 0.02 * 50^(j/5), j = 0..5, 8 per side x 6 x 6 = 576
    velocities, FP32 storage) to 1e-8 under a wall-clock cap."""
    from . import fdlb as F
    from . import workloads
    out = {}
    c1 = dict(nx=50, qx_half=4, qy=4, qz=4, kn=0.1, eta0=0.1, T_left=0.95, T_right=1.05, flow=F.FOURIER)
    s = F.Solver([F.Params(**c1)], device=device)
    sec, upd = _timed_steps(s, 5000)
    out["C1_single"] = {"steps": 5000, "seconds": sec, "updates_per_s": upd / sec, "us_per_step": 1e6 * sec / 5000,
                        "schedule": s.schedule()[0]}
    s.close()
    s = F.Solver([F.Params(**c1)] * 2048, device=device)
    s.step(50)
    sec, upd = _timed_steps(s, 500)
    out["C1_2048_replicas"] = {"steps": 500, "seconds": sec, "updates_per_s": upd / sec, "ms_per_step": 1e3 * sec / 500,
                               "schedule": s.schedule()[0]}
    s.close()
    # C2
    res = {}
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-8)):
        ps = [F.Params(**d) for d in workloads.couette_sweep(prec)]
        s = F.Solver(ps, device=device)
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            s.run(tol, 2_000_000, check_every=2000, timeout_s=c2_cap_s)
        except F.FdlbError:
            pass
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        _, st, n = s.status()
        res[prec] = {"tol": tol, "seconds": sec, "status": st.tolist(), "steps": n.tolist(),
                     "M": {i: s.moments(i) for i in range(s.count) if st[i] == F.CONVERGED},
                     "params": [(p.eta0, p.kn) for p in ps]}
        s.close()
    errs = []
    for i, M32 in res["fp32"]["M"].items():
        if i not in res["fp64"]["M"]:
            continue
        M64 = res["fp64"]["M"][i]
        errs.append({"eta0": res["fp32"]["params"][i][0], "kn": res["fp32"]["params"][i][1],
                     "n_rel": float(np.max(np.abs(M32["n"] - M64["n"]) / M64["n"])),
                     "T_rel": float(np.max(np.abs(M32["T"] - M64["T"]) / M64["T"])),
                     "uy_rel": float(np.max(np.abs(M32["uy"] - M64["uy"])) / np.max(np.abs(M64["uy"]))),
                     "Pxy_rel": float(np.max(np.abs(M32["Pxy"] - M64["Pxy"])) / np.max(np.abs(M64["Pxy"]))),
                     "steps_fp32_fp64": [res["fp32"]["steps"][i], res["fp64"]["steps"][i]]})
    out["C2"] = {k: {kk: vv for kk, vv in v.items() if kk not in ("M", "params")} for k, v in res.items()}
    out["C2"]["fp32_at_1e-8_vs_fp64_at_1e-10"] = errs
    # C3
    ps = []
    for eta in (0.05, 0.2, 0.35):
        for j in range(6):
            ps.append(F.Params(nx=400, qx_half=8, qy=6, qz=6, kn=0.02 * 50.0 ** (j / 5.0), eta0=eta, accel_y=0.05, grid="tanh",
                               stretch=1.5, flow=F.POISEUILLE, precision="fp32"))
    s = F.Solver(ps, device=device)
    sec, rc = _solve(s, F, c3_cap_s)
    out["C3"] = _summary(s, F, sec)
    out["C3"]["updates_per_s"] = out["C3"]["node_velocity_updates"] / sec
    _, st, n = s.status()
    out["C3"]["per_instance"] = [{"eta0": p.eta0, "kn": p.kn, "status": int(a), "steps": int(b)} for p, a, b in zip(ps, st, n)]
    s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=2048)
    ap.add_argument("--test", type=int, default=512)
    ap.add_argument("--cap-s", type=float, default=240.0)
    ap.add_argument("--test-cap-s", type=float, default=120.0)
    ap.add_argument("--plain-sample", type=int, default=8)
    ap.add_argument("--configs", action="store_true", help="run the named set-ups C1-C3 instead of the sweep study")
    a = ap.parse_args()
    if a.configs:
        print(json.dumps(configs()), flush=True)
    else:
        print(json.dumps(run(a.instances, a.test, a.cap_s, a.test_cap_s, a.plain_sample)), flush=True)


if __name__ == "__main__":
    main()
