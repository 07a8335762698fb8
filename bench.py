#!/usr/bin/env python
"""Benchmark of the GB300 FDLB solver on the Couette-flow parameter sweep.

Workload (the sweep the headline metric is quoted on): Couette flow, Nx = 200 nodes
tanh-stretched toward the walls (A = 1.5), walls at T = 1 moving at u_y = -0.42/+0.42,
eta0 in {0.1, 0.2, 0.3, 0.4} x Kn in {0.05, 0.1, 0.5} (12 instances in one batch),
velocities 12 half-range x (6 per side) x 6 x 4 full-range = 288 per node, f stored in
FP32 with FP64 moments/closure/residual.  Synthetic (no dataset): the uniform
equilibrium start of every instance.

Every RK3 step runs every row of the hot path: moments, chi, transport, gradients,
projected Shakhov + J1 target, WENO-5 advection with diffuse walls, RK3 combination,
per-step residual and status.  Instances that become non-finite (the scheme is linearly
unstable at eta0 >= 0.3 for this velocity set) are frozen by the status logic and do no
further work; the work count uses the per-instance step counters, so only performed
updates are counted.

One bench step = one steady-state solve of the whole sweep to residual 1e-8 (instances
freeze when they converge), warm-started from the profiles predicted by the warm-start
network (trained during set-up on 36 other Couette instances the solver itself solved).
value = node-velocity updates/s performed over the timed solves; steady_state_solves_per_s
= converged instances per second; batched_cold_start = the same solve from the uniform
start; plain_fp64_per_instance = every instance that converged, solved alone in FP64 storage,
one after another; cpu_baseline = the FP64 oracle on the host cores, one process per
instance.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fdlb|reference]

N > 1 runs under torchrun, one rank per GPU, each rank its own copy of the sweep (weak
scaling, no data-path collective; a barrier and a max-reduce of the time only).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "steady-state solves/s at residual 1e-8 (batched+warm-start vs plain FP64); node-vel updates/s, % BW"
UNIT = "node-velocity updates/s"
ETAS = (0.1, 0.2, 0.3, 0.4)
KNS = (0.05, 0.1, 0.5)
WORKLOAD = "Couette sweep: 12 instances (eta0 {0.1,0.2,0.3,0.4} x Kn {0.05,0.1,0.5}), Nx=200 tanh A=1.5, walls T=1 u_y=-+0.42, 12x6x4=288 velocities, FP32 storage"

# nominal peaks of the ALU pipes (152 SMs x lanes x 2 flops x 2.07 GHz max SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12      # 80.5
FP64_PEAK_TFLOPS = 1.25                                # recipe nominal (measured FMA probe: 1.22)
HBM_FALLBACK_GBS = 6800.0                              # recipe fallback when no measured copy rate exists
KERNEL_SRC = os.path.join(ROOT, "paper_2308_15407_gb300", "csrc", "fdlb_kernels.cu")
# ncu DRAM bytes (read + write) per k_update<float,float> launch on the 12-instance sweep,
# cold cache, mean over the three stages of one capture, with the SHA-256 prefix of the
# kernel source it was taken on; the bench reports it only while the source is unchanged.
UPDATE_TRAFFIC = {"bytes": 6691499, "kernel_src_sha16": "37dfbdfebdbecda5"}


def kernel_src_sha16():
    import hashlib
    with open(KERNEL_SRC, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of the GB300s, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "of measured (STREAM-style copy, read + write bytes)"
    except (OSError, KeyError, ValueError, TypeError):
        return HBM_FALLBACK_GBS, "of fallback (no measured peak available)"


def couette_params(F, precision="fp32"):
    return [F.Params(nx=200, qx_half=6, qy=6, qz=4, kn=kn, eta0=eta, U_left=-0.42, U_right=0.42, grid="tanh",
                     stretch=1.5, flow=F.COUETTE, precision=precision) for eta in ETAS for kn in KNS]


# ----------------------------------------------------------------------------- flop models
def kernel_flops(kind, p, nx, nvel):
    """Arithmetic per launch of one instance from the kernels' operation counts (FP64 flops;
    FP32 flops for the update of an FP32-storage instance).  The closure assumes the 8-point
    auxiliary rule, which the kernel uses whenever |u_x|/sqrt(T) < 0.02 and Q <= 12 (all
    nodes of these wall-bounded flows once the start-up transient has passed)."""
    Q, Qy, Qz = p.qx_half, p.qy, p.qz
    Tc = Qy * Qz if Qz else (2 * Qy if Qy else 2)
    if kind == "update":
        return (83 + (2 * Qy if p.accel_y else 0)) * nx * nvel
    if kind == "moments":
        per_node = 60 * Q + 120 if p.precision == "fp32" else 12 * nvel + 60 * Q + 120
        return per_node * nx
    if kind == "nodal":
        M = 8 if Q <= 12 else 16
        My = (Qy + 5) // 2 if Qy else 0
        Mz = (Qz + 5) // 2 if Qz else 0
        closure = 235
        xproj = 2 * M * (50 + 9 * Q) + 8 * Q * (M - 1) + 16 * Q * Q
        yz = My * (5 + 8 * Qy) + 4 * Qy * My + 8 * Qy * Qy
        if Qz:
            yz += Mz * (3 + 6 * Qz) + 3 * Qz * Mz + 6 * Qz * Qz
        assembly = 8 * Qy * 4 + 4 * Tc * 3
        return nx * (closure + xproj + yz + assembly)
    if kind == "resid":
        return 20 * nx
    return 0


def update_bytes_per_step(p, nx, nvel):
    """Algorithmic f traffic of the update kernel per RK3 step of one instance: 8 s per
    node-velocity (stage 1 reads f and writes f1; stages 2 and 3 read the stage value and the
    step's starting f and write), s = 4 B in FP32 storage, 8 B in FP64."""
    s = 4 if p.precision == "fp32" else 8
    return 8 * s * nx * nvel


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle timing
def cpu_model():
    """Host CPU model as the OS reports it (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def _oracle_worker(args):
    """One process: the oracle on one sweep instance for about `seconds` of RK3 steps
    (at least `min_steps`), single-threaded numpy.  Returns (steps, seconds, updates)."""
    eta, kn, seconds, min_steps = args
    sys.path.insert(0, ROOT)
    import numpy as np
    np.seterr(all="ignore")       # the eta0 >= 0.3 instances go non-finite (timed all the same)
    from oracle import fdlb as ofd
    p = ofd.Params(nx=200, qx_half=6, qy=6, qz=4, kn=kn, eta0=eta, U_left=-0.42, U_right=0.42, grid="tanh", stretch=1.5)
    o = ofd.Oracle(p)
    o.step(1)
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t0
        if n >= min_steps and el >= seconds:
            break
    return n, el, n * o.f.shape[0] * o.f.shape[1] * p.nx


def oracle_pool_rate(seconds=8.0, min_steps=1):
    """The FP64 oracle as it stands on instances of the sweep at once, one spawned process per
    instance (single-threaded numpy), as many instances as the host gives cores (at most the
    12, in sweep order): aggregate node-velocity updates/s = all processes' updates over the
    longest process's timed seconds (the timed windows run concurrently; process start-up and
    set-up are not timed)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    jobs = [(eta, kn, seconds, min_steps) for eta in ETAS for kn in KNS]
    procs = max(1, min(cores, len(jobs)))
    jobs = jobs[:procs]
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, jobs, chunksize=1)
    wall = max(r[1] for r in res)
    updates = sum(r[2] for r in res)
    steps = [r[0] for r in res]
    return {"rate": updates / wall, "wall": wall, "processes": procs, "host_cores": cores, "steps": steps,
            "cpu_model": cpu_model()}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times = []
    rates = []
    for _ in range(args.warmup):
        oracle_pool_rate(seconds=0.0, min_steps=1)
    last = None
    for _ in range(args.steps):
        last = oracle_pool_rate(seconds=8.0)
        times.append(last["wall"])
        rates.append(last["rate"])
    value = statistics.mean(rates)
    sample = (f"the first {last['processes']} instances of the sweep (200 nodes x 288 velocities each), one spawned "
              f"single-threaded process per instance, ~8 s of RK3 steps each ({min(last['steps'])}-{max(last['steps'])} steps); "
              f"CPU: {last['cpu_model']}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "bounded sample (see cpu_baseline.sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["processes"], "host_cores": last["host_cores"],
                         "cpu_model": last["cpu_model"], "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
TOL = 1e-8            # steady-state residual of one solve
MAX_STEPS = 200000    # per solve
CHECK = 2000          # steps between host checks of the instance status


def solve(s, F, nx, warm=None):
    """Reset every instance -- to the uniform start (n = 1, u = 0, T = 1), or to the local
    equilibrium of the warm-start network's profiles -- and solve to TOL."""
    import numpy as np
    if warm is not None:
        warm.apply(s)
    else:
        for i in range(s.count):
            s.set_profiles(i, np.ones(nx[i]), np.zeros(nx[i]), np.ones(nx[i]))
    try:
        s.run(TOL, MAX_STEPS, check_every=CHECK, timeout_s=600.0)
    except F.FdlbError as e:
        if e.code not in (F.FDLB_ENONFINITE, F.FDLB_EUNPHYSICAL):
            raise


def combine_ranks(dist, ms, updates, solved, device):
    """Whole-job totals of the timed region: the slowest rank's milliseconds (MAX over ranks)
    and the node-velocity updates and converged instances of all ranks (SUM); every rank
    receives them.  dist is None for a single process."""
    import torch
    if dist is None:
        return float(ms), float(updates), float(solved)
    tm = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    tu = torch.tensor([float(updates), float(solved)], dtype=torch.float64, device=device)
    dist.all_reduce(tu, op=dist.ReduceOp.SUM)
    return float(tm.item()), float(tu[0].item()), float(tu[1].item())


def run_fdlb(args):
    import numpy as np
    import torch
    from paper_2308_15407_gb300 import fdlb as F
    if not os.path.exists(F.LIB_PATH):
        from paper_2308_15407_gb300 import build
        build.build()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    params = couette_params(F, "fp32")
    stream = torch.cuda.current_stream()
    s = F.Solver(params, device=f"cuda:{local}", stream=stream)
    nx = s.nx
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{local}")   # 256 MB > 129 MB L2

    # ---- warm-start network (set-up, not timed): trained on steady states the solver produces
    # for 36 other Couette instances of the same family (eta0 0.05-0.25, Kn 0.03-0.5, U 0.3-0.5)
    from paper_2308_15407_gb300 import workloads
    from paper_2308_15407_gb300.warmstart import WarmStart
    t_setup = time.perf_counter()
    s_train = F.Solver([F.Params(**d) for d in workloads.couette_family(36, seed=23085)], device=f"cuda:{local}", stream=stream)
    try:
        s_train.run(TOL, MAX_STEPS, check_every=CHECK, timeout_s=600.0)
    except F.FdlbError as e:
        if e.code not in (F.FDLB_ENONFINITE, F.FDLB_EUNPHYSICAL):
            raise
    Xtr, Ytr = WarmStart.dataset(s_train)
    warm = WarmStart(max_points=Xtr.shape[0], seed=1, device=f"cuda:{local}")
    hist = warm.fit(Xtr, Ytr, steps=2000)
    s_train.close()
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup

    for _ in range(args.warmup):
        solve(s, F, nx, warm)
    torch.cuda.synchronize()

    # ---- timed region: K full warm-started steady-state solves of the sweep
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    updates = 0.0
    solved = 0
    steps_per_solve = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        for j in range(args.steps):
            flush.fill_(float(j))                      # evict L2 between timed iterations (not timed)
            torch.cuda.synchronize()
            ev[j][0].record(stream)
            solve(s, F, nx, warm)                     # network profiles -> set_profiles, fdlb_run to TOL
            ev[j][1].record(stream)
            _, status, done = s.status()
            updates += float(sum(int(d) * a * b for d, a, b in zip(done, nx, s.nvel)))
            solved += int((status == F.CONVERGED).sum())
            steps_per_solve.append([int(d) for d in done])
        torch.cuda.synchronize()
        barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    sched = "%s (cluster of %d CTAs available)" % s.schedule()
    ms_max, updates_all, solved_all = combine_ranks(dist, ms, updates, solved, f"cuda:{local}")
    value = updates_all / (ms_max * 1e-3)
    solves_per_s = solved_all / (ms_max * 1e-3)
    _, status, _ = s.status()

    # ---- kernel durations: 2000 steps of the sweep with the library's per-launch CUDA events
    # on its stream (launches one by one instead of replaying the step graph; same kernels)
    for i in range(s.count):
        s.set_profiles(i, np.ones(nx[i]), np.zeros(nx[i]), np.ones(nx[i]))
    s.step(600)                                        # past the start-up transient
    st0 = s.status()[2].copy()
    s.profile(True)
    PSTEPS = 2000
    s.step(PSTEPS)
    prof = s.profile_read()
    s.profile(False)
    pdone = s.status()[2] - st0
    total_kernel_ms = sum(v[0] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    kname = {"update": "k_update<float,float>", "moments": "k_moments<float>", "nodal": "k_nodal<8>", "resid": "k_resid"}
    upd_ms, upd_launches = prof["update"]
    # algorithmic work over the profiled steps: per instance, its steps done x per-step work
    upd_bytes = float(sum(update_bytes_per_step(params[i], nx[i], s.nvel[i]) * int(pdone[i]) for i in range(s.count)))
    upd_flops = float(sum(3 * kernel_flops("update", params[i], nx[i], s.nvel[i]) * int(pdone[i]) for i in range(s.count)))
    peak_gbs, peak_src = hbm_peak()
    achieved_gbs = upd_bytes / (upd_ms * 1e-3) / 1e9
    achieved_tflops = upd_flops / (upd_ms * 1e-3) / 1e12
    traffic = UPDATE_TRAFFIC["bytes"] if UPDATE_TRAFFIC["kernel_src_sha16"] == kernel_src_sha16() else None
    roofline = {"bound": "hbm", "kernel": kname["update"], "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                "frac": achieved_gbs / peak_gbs, "peak_source": peak_src,
                "traffic": traffic,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, cold cache, "
                                   "taken on the current kernel source" if traffic is not None else
                                   "no ncu capture of the current kernel source"),
                "algorithmic_bytes": "8 s per node-velocity and RK3 step (s = 4 B): stage 1 reads f and writes f1, "
                                     "stages 2 and 3 read the stage value and the step's f and write; "
                                     "%.0f B per launch on average" % (upd_bytes / max(1, upd_launches)),
                "alu": {"achieved": achieved_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved_tflops / FP32_PEAK_TFLOPS,
                        "peak_source": "nominal FP32: 152 SMs x 128 lanes x 2 x 2.07 GHz",
                        "flops": "83 FP32 flops per node-velocity and stage (update arithmetic, counted by hand)"},
                "dominant_kernel": kname[dom], "share": upd_ms / total_kernel_ms if total_kernel_ms else None,
                "launch_us": {k: 1e3 * v[0] / max(1, v[1]) for k, v in prof.items()},
                "kernel_ms_per_step": {k: v[0] / PSTEPS for k, v in prof.items()},
                "measured_over": "%d RK3 steps of the sweep after 600 start-up steps, per-launch CUDA events on the "
                                 "library's stream" % PSTEPS}
    # launches in the timed region: per solve, 4 per instance for the reset (profiles x2,
    # moments, residual anchor) and 7 per RK3 step of the batch (closure and update per stage,
    # residual) until the last instance stops (fdlb_run advances in chunks of CHECK steps)
    gpu_launches = sum(4 * s.count + 7 * CHECK * math.ceil(max(x) / CHECK) for x in steps_per_solve)

    # ---- throughput regime: the 2048-instance mixed sweep in one batch (f > L2)
    batch = None
    if rank == 0:
        sdicts = workloads.batched_sweep()
        sp = [F.Params(**d) for d in sdicts]
        sw = F.Solver(sp, device=f"cuda:{local}", stream=stream)
        sw.step(48)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = sw.status()[2].copy()
        b0.record(stream)
        sw.step(160)
        b1.record(stream)
        torch.cuda.synchronize()
        bms = b0.elapsed_time(b1)
        bdone = sw.status()[2] - n0
        bupd = float(sum(int(d) * a * b for d, a, b in zip(bdone, sw.nx, sw.nvel)))
        sw.profile(True)
        m0 = sw.status()[2].copy()
        sw.step(32)
        bprof = sw.profile_read()
        sw.profile(False)
        mdone = sw.status()[2] - m0
        f_bytes = sum(sw.nx[i] * sw.nvel[i] * 4 for i in range(sw.count))
        ub = float(sum(update_bytes_per_step(sp[i], sw.nx[i], sw.nvel[i]) * int(mdone[i]) for i in range(sw.count)))
        ugbs = ub / (bprof["update"][0] * 1e-3) / 1e9
        bdom = max(bprof, key=lambda k: bprof[k][0])
        bflops = sum(kernel_flops("nodal", sp[i], sw.nx[i], sw.nvel[i]) * 3 * int(mdone[i]) for i in range(sw.count))
        nach = bflops / (bprof["nodal"][0] * 1e-3) / 1e12
        batch = {"workload": "2048 instances: flow, nx 32..512, Q_x^h 4..8, Kn, eta0 drawn (seed 23084); reduced velocity sets; FP32 storage",
                 "f_bytes": f_bytes, "active_instances": int((sw.status()[1] == F.ACTIVE).sum()),
                 "updates_per_s": bupd / (bms * 1e-3), "ms_per_rk3_step": bms / 160,
                 "kernel_ms_per_step": {k: v[0] / 32 for k, v in bprof.items()},
                 "dominant_kernel": kname[bdom],
                 "update_hbm": {"achieved_gbs": ugbs, "peak_gbs": peak_gbs, "frac": ugbs / peak_gbs,
                                "bytes": "8 s per node-velocity and RK3 step, s = 4 B"},
                 "nodal_alu": {"achieved_tflops": nach, "frac_of_fp64_nominal": nach / FP64_PEAK_TFLOPS,
                               "flops": "hand count of the closure's operations (kernel_flops)"}}
        sw.close()

    # ---- e2e: the timed solve again through the public API with host buffers: features on
    # the host -> device, network prediction -> host, profiles -> device (set_profiles),
    # fdlb_run to TOL, moments -> host; host wall clock
    e2e = None
    if rank == 0:
        flush.fill_(0.5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solve(s, F, nx, warm)
        outs = [s.moments(i) for i in range(s.count)]                                  # device -> host
        el = time.perf_counter() - t0
        _, st_e, done_e = s.status()
        e2e = {"value": float(sum(int(d) * a * b for d, a, b in zip(done_e, nx, s.nvel))) / el, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(16 * 4 * n + 4 * ((n + 31) // 32 * 32) * 8 for n in nx)),
               "d2h_bytes_per_step": int(sum(3 * 4 * n + 8 * 8 * n for n in nx)),
               "solves_per_s": float((st_e == F.CONVERGED).sum()) / el,
               "what": "the warm-started solve of the timed region, host clock, host buffers in and out"}

    # ---- the same batched solve from the uniform start (no warm start), once
    cold = None
    cold_moments = {}
    if rank == 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(0.25)
        torch.cuda.synchronize()
        e0.record(stream)
        solve(s, F, nx)
        e1.record(stream)
        torch.cuda.synchronize()
        _, st_c, done_c = s.status()
        sec = e0.elapsed_time(e1) * 1e-3
        cold = {"solves_per_s": float((st_c == F.CONVERGED).sum()) / sec, "seconds": sec,
                "rk3_steps_per_instance": [int(d) for d in done_c]}
        cold_moments = {i: s.moments(i) for i in range(s.count) if st_c[i] == F.CONVERGED}

    # ---- plain FP64 per-instance solver: every instance that converged in the timed solves,
    # solved alone in FP64 storage from the uniform start, one after another
    plain = None
    if rank == 0:
        conv = [i for i in range(s.count) if status[i] == F.CONVERGED]
        tot = 0.0
        per = []
        errs = []
        for i in conv:
            p64 = F.Params(**{**params[i].__dict__, "precision": "fp64"})
            s64 = F.Solver([p64], device=f"cuda:{local}", stream=stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s64.run(TOL, MAX_STEPS, check_every=CHECK, timeout_s=600.0)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            tot += sec
            n64 = int(s64.status()[2][0])
            per.append({"eta0": params[i].eta0, "kn": params[i].kn, "steps": n64, "seconds": sec})
            if i in cold_moments:
                M32, M64 = cold_moments[i], s64.moments(0)
                errs.append({"eta0": params[i].eta0, "kn": params[i].kn,
                             "n_rel": float(np.max(np.abs(M32["n"] - M64["n"]) / M64["n"])),
                             "T_rel": float(np.max(np.abs(M32["T"] - M64["T"]) / M64["T"])),
                             "uy_rel": float(np.max(np.abs(M32["uy"] - M64["uy"])) / np.max(np.abs(M64["uy"]))),
                             "Pxy_rel": float(np.max(np.abs(M32["Pxy"] - M64["Pxy"])) / np.max(np.abs(M64["Pxy"]))),
                             "steps_fp32_fp64": [int(cold["rk3_steps_per_instance"][i]), n64]})
            s64.close()
        worst = {k: max(e[k] for e in errs) for k in ("n_rel", "T_rel", "uy_rel", "Pxy_rel")} if errs else None
        plain = {"solves_per_s": len(conv) / tot if tot else None, "instances": len(conv), "seconds": tot,
                 "per_instance": per,
                 "what": "each instance that converged in the timed solves, alone in FP64 storage from the uniform "
                         "start, solved to residual %g one after another" % TOL,
                 "fp32_vs_fp64_profiles": {"what": "batched FP32-storage cold solve vs the plain FP64 solve of the "
                                                   "same instance, both at residual %g" % TOL,
                                           "worst": worst, "per_instance": errs}}

    # ---- CPU baseline (rank 0, N = 1 only): the oracle on all host cores, one process per
    # instance of the sweep
    cpu = None
    if rank == 0 and world == 1:
        r = oracle_pool_rate(seconds=10.0)
        cpu = {"value": r["rate"], "unit": UNIT, "cores": r["processes"], "host_cores": r["host_cores"],
               "cpu_model": r["cpu_model"], "kind": "oracle",
               "sample": "the first %d instances of the sweep (200 nodes x 288 velocities), one spawned single-threaded "
                         "numpy process per instance, ~10 s of FP64 RK3 steps each (%d-%d steps)"
                         % (r["processes"], min(r["steps"]), max(r["steps"]))}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instances_per_gpu": len(params),
                       "bench_step": f"one steady-state solve of the sweep to residual {TOL:g} (per-instance freezing), warm-started from the network's profiles",
                       "precision": "f stored/advected in FP32; moment sums and velocity projections in double-float (FP32 pairs, ~1e-14); closure chain, moment finalisation and residual FP64",
                       "schedule": sched,
                       "l2": "flushed between timed iterations (256 MB write)",
                       "instances_converged_per_solve": int(solved / max(1, args.steps)),
                       "instances_failed_nonfinite": int((status == F.FAILED_NONFINITE).sum()),
                       "rk3_steps_per_instance_last_solve": steps_per_solve[-1] if steps_per_solve else None,
                       "parallelism": f"instance replicas x{world}"},
            "steady_state_solves_per_s": solves_per_s,
            "warm_start": {"train_instances": int(len(Xtr) // 200), "train_points": int(Xtr.shape[0]),
                           "loss_first_last": [hist[0], hist[-1]], "setup_seconds": t_setup,
                           "network": "16 -> 4x128 GELU -> 3, tcgen05 BF16/FP32, full-batch Adam 2000 steps"},
            "batched_cold_start": cold,
            "throughput_regime": batch,
            "plain_fp64_per_instance": plain,
            "solves_per_s_vs_plain_fp64": (solves_per_s / plain["solves_per_s"]) if plain and plain["solves_per_s"] else None,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(gpu_launches),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_profile_case(case, precision):
    """Small fixed workloads for ncu captures (no timing, no JSON line).
    couette1 / couette12: one instance (eta0 = 0.2, Kn = 0.5) or the whole Couette sweep;
    sweep2048: the 2048-instance mixed sweep (f 162 MB in FP32); tiled schedule: creation
    (5 launches), 20 steps (7 launches each), 3 more steps.
    mlp: the warm-start network on 32768 points, 6 training steps and one prediction."""
    import torch
    from paper_2308_15407_gb300 import fdlb as F
    if not os.path.exists(F.LIB_PATH):
        from paper_2308_15407_gb300 import build
        build.build()
    if case == "mlp":
        P = 32768
        g = torch.Generator(device="cuda").manual_seed(5)
        X = torch.randn(P, 16, device="cuda", generator=g) * 0.5
        Y = torch.randn(P, 3, device="cuda", generator=g) * 0.1
        net = F.MLP(max_points=P, seed=1)
        for _ in range(6):
            net.train_step(X, Y, 1e-3)
        net.predict(X)
        torch.cuda.synchronize()
        print("ok")
        return
    if case == "sweep2048":
        from paper_2308_15407_gb300 import workloads
        ps = [F.Params(**d) for d in workloads.batched_sweep(precision=precision)]
    else:
        ps = couette_params(F, precision)
    if case == "couette1":
        ps = ps[4:5]
    s = F.Solver(ps)
    s.set_schedule("tiled")
    s.step(20)
    torch.cuda.synchronize()
    s.step(3)
    torch.cuda.synchronize()
    print("ok")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fdlb", choices=["fdlb", "reference"])
    ap.add_argument("--profile-case", choices=["couette1", "couette12", "sweep2048", "mlp"], default=None,
                    help="run a small fixed workload for an ncu capture instead of the benchmark")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case, args.precision)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_fdlb(args)


if __name__ == "__main__":
    main()
