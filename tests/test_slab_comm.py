"""The transports of the slab decomposition on CPU (no GPU): the reductions
and the halo exchange that a decomposed step hands to its caller.

  * TorchComm over two and three gloo ranks: max, min and sum of host
    buffers equal the single-rank reductions of all ranks' buffers (the sum
    in rank order, identical on every rank); the exchange delivers each
    neighbour's rows, with and without the periodic wrap.
  * LocalComm over threads: the same checks, and a slab that stops calling
    makes the others fail within the timeout instead of hanging.
"""
import os
import socket
import sys
import threading

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _buffers(rank, n=7):
    r = np.random.default_rng(1000 + rank)
    return r.normal(size=n) * 10.0 ** r.integers(-3, 4, size=n)


def _rows(rank, side, n=12):
    """the rows a rank sends below (side 0) or above (side 1)"""
    return 1000.0 * rank + 100.0 * side + np.arange(n, dtype=np.float64)


def _check_rank(comm, rank, world, periodic):
    from paper_2107_12027_gb300 import esmm
    out = {}
    for op, name in ((esmm.OP_MAX, "max"), (esmm.OP_MIN, "min"), (esmm.OP_SUM, "sum")):
        buf = _buffers(rank)
        comm.allreduce(buf, op)
        out[name] = buf
    n = 12
    has_lo = periodic or rank > 0
    has_hi = periodic or rank < world - 1
    rl = np.full(n, np.nan) if has_lo else None
    rh = np.full(n, np.nan) if has_hi else None
    comm.exchange(_rows(rank, 0) if has_lo else None, _rows(rank, 1) if has_hi else None, rl, rh)
    out["recv_lo"], out["recv_hi"] = rl, rh
    return out


def _expected(world):
    bufs = [_buffers(r) for r in range(world)]
    s = bufs[0].copy()
    for b in bufs[1:]:
        s = s + b
    return {"max": np.max(bufs, axis=0), "min": np.min(bufs, axis=0), "sum": s}


def _verify(res, world, periodic):
    exp = _expected(world)
    for rank in range(world):
        got = res[rank]
        for k in ("max", "min", "sum"):
            assert np.array_equal(got[k], exp[k]), (rank, k)
        if periodic or rank > 0:
            assert np.array_equal(got["recv_lo"], _rows((rank - 1) % world, 1)), rank
        else:
            assert got["recv_lo"] is None
        if periodic or rank < world - 1:
            assert np.array_equal(got["recv_hi"], _rows((rank + 1) % world, 0)), rank
        else:
            assert got["recv_hi"] is None


def _torch_rank(rank, world, port, periodic, out):
    import datetime

    import torch.distributed as dist
    from paper_2107_12027_gb300.comm import TorchComm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        out[rank] = _check_rank(TorchComm(), rank, world, periodic)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, False), (2, True), (3, True)])
def test_torch_comm_gloo_ranks(world, periodic):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_torch_rank, args=(world, _free_port(), periodic, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == list(range(world))
    _verify(res, world, periodic)


@pytest.mark.parametrize("world,periodic", [(2, False), (3, True), (4, False)])
def test_local_comm_threads(world, periodic):
    from paper_2107_12027_gb300.comm import LocalComm
    lc = LocalComm(world, timeout=20.0)
    res = {}

    def run(r):
        res[r] = _check_rank(lc.rank(r), r, world, periodic)
    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    _verify(res, world, periodic)


def test_local_comm_times_out_instead_of_hanging():
    from paper_2107_12027_gb300 import esmm
    from paper_2107_12027_gb300.comm import LocalComm
    lc = LocalComm(2, timeout=0.5)
    with pytest.raises(threading.BrokenBarrierError):
        lc.rank(0).allreduce(np.zeros(3), esmm.OP_MAX)      # slab 1 never calls
