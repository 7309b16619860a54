"""Multi-process path of bench.py on CPU (gloo, world size 2): the replicas'
whole-job rate is the units all ranks processed over the slowest rank's time,
and every rank draws its own workload seed."""
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


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = [300.0, 500.0][rank]
    seconds = [2.0, 5.0][rank]
    out[rank] = (bench.job_throughput(dist, units, seconds), bench.reduce_max(dist, seconds, "cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a multi-threaded process
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        rate, tmax = res[rank]
        assert rate == pytest.approx(800.0 / 5.0)
        assert tmax == 5.0


def test_single_process_rate_and_per_rank_seeds():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(None, 300.0, 2.0) == 150.0
    p0, _ = bench.workload("small", 0)
    p1, _ = bench.workload("small", 1)
    assert p0.seed != p1.seed
