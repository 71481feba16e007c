"""Replica aggregation of bench.py on CPU: two gloo ranks report different step times; both
must see the slowest rank's time and the whole-job rate of both ranks' work."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
        ms, value = bench.job_rate(ms_local, world, 2.0e12, "cpu")
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_counts_all_work():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 150.0
        assert value == pytest.approx(2.0e12 * world / 0.150 / 1e9)


def test_job_rate_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.job_rate(80.0, 1, 1.0e12, "cpu")
    assert ms == 80.0 and value == pytest.approx(1.0e12 / 0.080 / 1e9)
