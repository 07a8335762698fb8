"""The multi-process path of bench.py on CPU ranks (gloo, world size 2): the whole-job totals
(slowest rank's time, summed work) and the rank-0-only reference arm.  Instances are
independent, so ranks exchange nothing but these timings."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [1200.0, 1500.0][rank]
        updates = [3.0e9, 5.0e9][rank]
        solved = [6, 5][rank]
        q.put((rank, bench.combine_ranks(dist, ms, updates, solved, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_combine_ranks_gloo_world_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = dict(q.get(timeout=10) for _ in range(2))
    for r in (0, 1):
        assert got[r] == (1500.0, 8.0e9, 11.0)        # MAX of times, SUM of work, on every rank


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(None, 10.0, 2.0e6, 3, "cpu") == (10.0, 2.0e6, 3.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_pool_rate", lambda **kw: called.append(kw))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(type("A", (), dict(steps=3, warmup=3, gpus=2))())
    assert buf.getvalue() == "" and not called
