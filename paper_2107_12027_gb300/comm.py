"""Transports for the slabs of a decomposed grid (esmm.Slab).

The library hands every reduction and halo exchange of a decomposed step to
its caller as host buffers (include/esmm.h, esmm_comm).  Two transports:

  * LocalComm: the slabs of one process, each driven by its own host thread
    (one GPU, or several GPUs of one process).  Threads meet at a barrier;
    no kernel waits on another.
  * TorchComm: one slab per rank of torch.distributed (gloo or any backend
    that reduces CPU tensors).

Both implement the same two calls: allreduce(buf, op) combines a float64
buffer in place over all slabs (op: esmm.OP_MAX, OP_MIN, OP_SUM), and
exchange(send_lo, send_hi, recv_lo, recv_hi) sends to the slab below and
above and receives theirs (None where there is no neighbour).  Slab s's
neighbours are s - 1 and s + 1, modulo the slab count (the library passes
None across a non-periodic end).
"""
from __future__ import annotations

import threading

import numpy as np

from . import esmm

_NP_OPS = {esmm.OP_MAX: np.maximum, esmm.OP_MIN: np.minimum, esmm.OP_SUM: np.add}


class LocalComm:
    """Shared state of nslab slabs in one process; ``rank(s)`` is slab s's
    transport.  Every wait is bounded (timeout seconds): a slab that stops
    calling makes the others' next call fail instead of hang."""

    def __init__(self, nslab, timeout=120.0):
        self.n = nslab
        self.timeout = timeout
        self.barrier = threading.Barrier(nslab, timeout=timeout)
        self.bufs = [None] * nslab

    def rank(self, s):
        return _LocalRank(self, s)


class _LocalRank:
    def __init__(self, shared, s):
        self.sh, self.s = shared, s

    def allreduce(self, buf, op):
        sh = self.sh
        sh.bufs[self.s] = buf.copy()
        sh.barrier.wait()
        acc = sh.bufs[0].copy()            # in slab order: the same result on every slab
        for b in sh.bufs[1:]:
            acc = _NP_OPS[op](acc, b)
        sh.barrier.wait()                  # every slab has read before the next call writes
        buf[:] = acc

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        sh = self.sh
        sh.bufs[self.s] = (None if send_lo is None else send_lo.copy(), None if send_hi is None else send_hi.copy())
        sh.barrier.wait()
        if recv_lo is not None:
            recv_lo[:] = sh.bufs[(self.s - 1) % sh.n][1]
        if recv_hi is not None:
            recv_hi[:] = sh.bufs[(self.s + 1) % sh.n][0]
        sh.barrier.wait()


class TorchComm:
    """The slabs as torch.distributed ranks (slab = rank).  Buffers travel
    as CPU tensors, so a gloo process group carries them (an NCCL job can
    pass a gloo group made with torch.distributed.new_group)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def allreduce(self, buf, op):
        import torch
        d = self.dist
        t = torch.from_numpy(np.ascontiguousarray(buf))
        rop = {esmm.OP_MAX: d.ReduceOp.MAX, esmm.OP_MIN: d.ReduceOp.MIN, esmm.OP_SUM: d.ReduceOp.SUM}[op]
        if op == esmm.OP_SUM:
            # a fixed order of the sum, the same on every rank: gather, add in rank order
            parts = [torch.empty_like(t) for _ in range(self.size)]
            d.all_gather(parts, t, group=self.group)
            acc = parts[0].clone()
            for q in parts[1:]:
                acc += q
            t = acc
        else:
            d.all_reduce(t, op=rop, group=self.group)
        buf[:] = t.numpy()

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        import torch
        n = next(len(a) for a in (send_lo, send_hi, recv_lo, recv_hi) if a is not None)
        mine = torch.zeros(2 * n, dtype=torch.float64)
        if send_lo is not None:
            mine[:n] = torch.from_numpy(send_lo)
        if send_hi is not None:
            mine[n:] = torch.from_numpy(send_hi)
        parts = [torch.empty_like(mine) for _ in range(self.size)]
        self.dist.all_gather(parts, mine, group=self.group)
        if recv_lo is not None:
            recv_lo[:] = parts[(self.rank - 1) % self.size][n:].numpy()
        if recv_hi is not None:
            recv_hi[:] = parts[(self.rank + 1) % self.size][:n].numpy()
