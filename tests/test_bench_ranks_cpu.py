"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
job's time is the slowest rank's, and the job's value counts every rank's
units (replicas: each rank analyses its own copy of the workload)."""
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    job = bench.job_time_ms(ms, world, "cpu")
    out[rank] = (job, bench.job_value(1000, world, 4, job))
    dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_value_counts_all_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        job, value = res[r]
        assert job == 15.0
        assert abs(value - 1000 * 2 * 4 / 0.015) < 1e-6


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(7.5, 1, "cpu") == 7.5
    assert bench.job_value(10, 1, 2, 1000.0) == 20.0
