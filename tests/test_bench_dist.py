"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its
own seeded problem; the job time is the slowest rank's and the rate counts
every rank's nodes (weak scaling)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        local_ms = 10.0 * (rank + 1)                      # rank 1 is the slower one
        job_ms = bench.job_time_ms(local_ms, w, dist, "cpu")
        x, prim = bench.workload(16, r)
        out[rank] = (r, w, lr, job_ms, bench.job_rate(16 * 16, 5, w, job_ms), float(prim[0].sum()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_rate():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, lr, job_ms, rate, _) in res.items():
        assert (r, w, lr) == (rank, world, rank)
        assert job_ms == 20.0                             # the slowest rank's time on every rank
        assert rate == pytest.approx(world * 256 * 3 * 5 / 0.020)
    # each rank has its own seeded problem
    assert res[0][5] != res[1][5]


def test_single_rank_needs_no_collective():
    import bench
    assert bench.job_time_ms(12.5, 1, None, "cpu") == 12.5
    assert bench.job_rate(100, 4, 1, 1000.0) == pytest.approx(100 * 3 * 4 / 1.0)
    x0, p0 = bench.workload(16, 0)
    x1, p1 = bench.workload(16, 0)
    assert np.array_equal(p0, p1)                         # seeded: the same problem again
