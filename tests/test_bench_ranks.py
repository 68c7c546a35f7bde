"""The multi-process path of bench.py on CPU: two gloo ranks (127.0.0.1)
agree on the slowest rank's time, and the whole-job rate counts the steps of
every rank over that time (replicas: one independent problem per GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(dist, times[rank], "cpu")
        out[rank] = (m, bench.job_rate(world, 10, m))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    world, times = 2, [120.0, 80.0]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), times, out), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        m, rate = out[rank]
        assert m == 120.0
        assert rate == pytest.approx(2 * 10 / 0.120)


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(None, 5.0, "cpu") == 5.0
    assert bench.job_rate(1, 30, 300.0) == pytest.approx(100.0)
