"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its own replica of the
batch, agree on the slowest rank's time, and the job's throughput counts every rank's rows
(weak scaling, no collective on the data path).  No GPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], world)
        out[rank] = (ms, bench.job_throughput(1000, 10, world, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_every_rank():
    world, port = 2, _free_port()
    times = [12.5, 20.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, times, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 20.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1) == 7.0
    assert bench.job_throughput(100, 4, 1, 2.0) == pytest.approx(100 * 4 / 0.002)
