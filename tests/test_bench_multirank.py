"""The multi-rank path of bench.py on the CPU: two gloo ranks agree on the slowest rank's time
and report the whole job's rate (every rank processes its own replica: weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.reduce_max(0.2 + 0.1 * rank, dist, "cpu")        # rank 1 is the slowest
        rate = bench.whole_job_rate(1.2e10, world, t)
        out[rank] = (t, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_max_time_and_whole_job_rate():
    world, port = 2, _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        t, rate = out[r]
        assert abs(t - 0.3) < 1e-12
        assert abs(rate - 2 * 1.2e10 / 0.3) < 1.0


def test_single_process_needs_no_collective():
    import bench
    assert bench.reduce_max(1.25) == 1.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
