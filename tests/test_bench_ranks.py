"""The replica (N > 1) host logic of bench.py on CPU with gloo, world size 2:
the job time is the maximum over ranks, the job rate counts every rank's
work over that time, and the reference arm runs on rank 0 only."""
from __future__ import annotations

import importlib.util
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    sys.path.insert(0, ROOT)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        # rank r took (10 + r) ms for the timed steps and (3 + 2r) ms end to end
        tmax, e2e = b.reduce_max_over_ranks([10.0 + rank, 3.0 + 2 * rank], world)
        rate = b.job_rate(world, 10, 100, tmax)
        ref = b.run_reference(type("A", (), {"workload": "cp", "warmup": 0, "steps": 1})(),
                              rank, world) if rank == 1 else "skipped"
        q.put((rank, tmax, e2e, rate, ref))
    finally:
        dist.destroy_process_group()


def test_replica_timing_max_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict((r, (t, e, rate, ref)) for r, t, e, rate, ref in (q.get() for _ in range(2)))
    for r in (0, 1):
        t, e, rate, _ = got[r]
        assert t == 11.0 and e == 5.0                   # the slowest rank on both ranks
        assert rate == pytest.approx(2 * 10 * 100 / 0.011)
    assert got[1][3] is None                            # reference arm: rank 0 only
