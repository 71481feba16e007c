"""Host logic of bench.py on CPU: replica aggregation (two gloo ranks report different step
times; both must see the slowest rank's time and the whole-job rate of both ranks' work)
and the algorithmic byte model behind the roofline."""
import os
import socket

import numpy as np

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
    # the manager's server process is started by spawn as well: a fork of this
    # (multi-threaded) interpreter may deadlock
    with mp.get_context("spawn").Manager() as m:
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


def _levels(m):
    """Pairs per binary-TT level for m sub-diagonal tiles (distance 1, 2, 4, ...)."""
    out, step = [], 1
    while step <= m:
        out.append((m - step) // (2 * step) + 1)
        step *= 2
    return out


def test_tensor_core_byte_model_counts_bulk_columns_and_every_launch():
    import bench
    rng = np.random.default_rng(0)
    for tree in ("binary_tt", "flat_ts"):
        n, nb = 12, 64
        dec = (rng.random(n) < 0.3).astype(int)
        got = bench.step_tc_bytes(dec, n, nb, tree, 0)
        want = {}
        for k in range(n):
            m = n - 1 - k
            cols = (m - 1) * nb                      # columns >= k+2
            if cols <= 0:
                continue
            A = 4.0 * nb * nb
            if dec[k] == 1:
                want["k_tc_lu_apply"] = want.get("k_tc_lu_apply", 0.0) + 4.0 * nb * cols * 2 + A
                rows = m * nb
                want["k_tc_lu_gemm"] = want.get("k_tc_lu_gemm", 0.0) + 4.0 * (
                    rows * nb + nb * cols + 2 * rows * cols)
                continue
            singles = m + 1 if tree == "binary_tt" else 1
            pairs = sum(_levels(m)) if tree == "binary_tt" else m
            kind = "tt" if tree == "binary_tt" else "ts"
            for role, per, cnt in (("unmqr_w", 8, singles), ("unmqr_c", 12, singles),
                                   (kind + "mqr_w", 12, pairs), (kind + "mqr_c1", 12, pairs),
                                   (kind + "mqr_c2", 12, pairs)):
                key = "k_tc_" + role
                want[key] = want.get(key, 0.0) + cnt * (per * nb * cols + A)
        assert set(got) == set(want)
        for key in want:
            assert got[key] == pytest.approx(want[key], rel=1e-12), key
