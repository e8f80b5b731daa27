"""Multi-process host logic of the benchmark on CPU (gloo, world size 2):
each rank runs its own replicas (no data-path collective), the job time is
the slowest rank's, and the rate is all ranks' cell-updates over it."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seconds = [2.0, 3.5][rank]                 # rank 1 is slower
        units = 1000.0
        t = bench.max_over_ranks(seconds, dist, "cpu")
        rate = bench.whole_job_rate(units, world, t)
        dist.barrier()
        q.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_time_and_weak_scaling_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, t, rate in res:
        assert t == 3.5
        assert rate == pytest.approx(2 * 1000.0 / 3.5)


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
