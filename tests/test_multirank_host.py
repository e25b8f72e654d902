"""The benchmark's multi-rank host logic on CPU: two gloo ranks, the slowest rank's time
decides, and the whole-job rate counts every rank's units (replicas, weak scaling)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        t = [2.0, 3.0][rank]                     # rank 1 is the slower one
        q.put((rank, bench.reduce_max(t, dist), bench.whole_job_rate(600.0, t, dist)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, tmax, rate in res:
        assert tmax == 3.0
        assert rate == pytest.approx(2 * 600.0 / 3.0)


def test_single_process_rate_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(1.5) == 1.5
    assert bench.whole_job_rate(10.0, 2.0) == 5.0
