"""The multi-GPU path of the benchmark runs independent replicas (the
method does not shard without the paper's ghost exchange): each rank times
its own copy of the step, and the only collective is one all-reduce of the
step time (maximum over ranks).  Checked here with two gloo ranks on CPU."""
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


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms_max, value = bench.replica_throughput(ms, 1_000_000, world, torch.device("cpu"))
        q.put((rank, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_the_whole_job():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in out:
        assert ms_max == pytest.approx(15.0)  # every rank agrees on the maximum
        assert value == pytest.approx(2 * 1_000_000 / 0.015)  # all ranks' units over the slowest time


def test_one_replica_needs_no_process_group():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    ms_max, value = bench.replica_throughput(4.0, 1000, 1, torch.device("cpu"))
    assert ms_max == 4.0 and value == pytest.approx(1000 / 0.004)
