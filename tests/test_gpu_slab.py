"""Slab decomposition on one GPU: a grid split along its second index into 2
or 3 slabs, each a handle of its own driven by its own host thread and CUDA
stream, with the reductions and halo exchanges of every step going through
LocalComm (host buffers; no kernel waits on another).  Against the same grid
undecomposed, through the C ABI:

  * the right-hand side of each slab's held rows equals the whole grid's on
    its own rows, bit for bit;
  * three SSP-RK3 steps with the adaptive mesh and the eq. cfl step leave
    every slab's own rows of cons, J and x, and every step size, equal to
    the undecomposed run's bit for bit with an outflow second direction
    (RHD in both forms, RMHD).  Across a periodic seam the halo rows hold
    x_2 minus or plus the period, and the redundant mesh iteration on them
    rounds differently from the owner's (the whole grid adds the period
    only where it reads a ghost), so there the own rows agree to rounding
    (1e-12 relative); with a static mesh they are bitwise again;
  * the totals (a sum over slabs) agree to rounding.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl
from paper_2107_12027_gb300.comm import LocalComm

pytestmark = pytest.mark.gpu


def _case(kind, nx, ny):
    if kind == "riemann":
        lo, hi, bc = (-1.0, -1.0), (1.0, 1.0), (esmm.OUTFLOW, esmm.OUTFLOW)
        x = wl.random_mesh(nx, ny, wl.rng(601), amp=0.15, lo=lo, hi=hi, periodic=(False, False))
        prim = wl.quadrant_riemann(x, wl.quadrant_states(wl.rng(602), vmax=0.5), split=(0.1, -0.15))
        return lo, hi, bc, x, prim, dict(alpha=1200.0)
    if kind == "smooth":
        lo, hi, bc = (0.0, 0.0), (1.0, 1.0), (esmm.PERIODIC, esmm.PERIODIC)
        x = wl.wavy_mesh(nx, ny, amp=0.04)
        return lo, hi, bc, x, wl.smooth_random_state(x, wl.rng(603)), dict(alpha=20.0)
    lo, hi, bc = (-0.5, -0.5), (0.5, 0.5), (esmm.OUTFLOW, esmm.OUTFLOW)
    x = wl.uniform_mesh(nx, ny, lo, hi, periodic=(False, False))
    return lo, hi, bc, x, wl.rotor(x), dict(alpha=800.0)


def _grid_kw(kind, form):
    kw = dict(p=2, w=5, precision=esmm.MIXED if form == "mixed" else esmm.FP64, monitor=esmm.MONITOR_LNRHO)
    if kind == "rotor":
        kw.update(phys=esmm.RMHD, gamma=4.0 / 3.0)
    return kw


def _slabs(nslab, n, lo, hi, bc, prim, x, steps, kw):
    import torch
    comm = LocalComm(nslab, timeout=120.0)
    out = {}

    def run(s):
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        with esmm.Slab(n, nslab, s, comm.rank(s), lo=lo, hi=hi, bc=bc, stream=st.cuda_stream, **kw) as g:
            g.state_set(prim, x)
            tot0 = g.totals()
            dts = [g.rk_step() for _ in range(steps)]
            out[s] = dict(dts=dts, own=(g.own0, g.own1), tot0=tot0, tot=g.totals(),
                          cons=g.state_get(esmm.GET_CONS), J=g.state_get(esmm.GET_J), x=g.state_get(esmm.GET_X))
    with ThreadPoolExecutor(nslab) as ex:
        for f in [ex.submit(run, s) for s in range(nslab)]:
            f.result()
    return out


CASES = [("riemann", 48, 80, 2, "fp64"), ("smooth", 40, 96, 3, "fp64"), ("riemann", 40, 66, 2, "mixed"),
         ("rotor", 48, 64, 2, "fp64"), ("riemann", 40, 99, 3, "fp64")]


@pytest.mark.parametrize("kind,nx,ny,nslab,form", CASES)
def test_slabs_step_bitwise_as_the_whole_grid(kind, nx, ny, nslab, form):
    lo, hi, bc, x, prim, extra = _case(kind, nx, ny)
    kw = dict(_grid_kw(kind, form), **extra)
    steps = 3
    with esmm.Grid((nx, ny), lo, hi, bc=bc, **kw) as g:
        g.state_set(prim, x)
        tot0 = g.totals()
        dts = [g.rk_step() for _ in range(steps)]
        ref = dict(cons=g.state_get(esmm.GET_CONS), J=g.state_get(esmm.GET_J), x=g.state_get(esmm.GET_X),
                   tot=g.totals())
    out = _slabs(nslab, (nx, ny), lo, hi, bc, prim, x, steps, kw)
    rows = []
    seam = bc[1] == esmm.PERIODIC

    def same(u, v):
        if not seam:
            return np.array_equal(u, v)
        return np.abs(u - v).max() <= 1e-12 * np.abs(v).max()
    for s in range(nslab):
        o = out[s]
        a, b = o["own"]
        rows.append((a, b))
        if seam:
            assert np.allclose(o["dts"], dts, rtol=1e-12, atol=0), (s, o["dts"], dts)
        else:
            assert o["dts"] == dts, (s, o["dts"], dts)
        assert same(o["cons"], ref["cons"][:, a:b]), s
        assert same(o["J"], ref["J"][a:b]), s
        assert same(o["x"], ref["x"][:, a:b]), s
        assert np.allclose(o["tot0"], tot0, rtol=1e-13, atol=0)
        assert np.allclose(o["tot"], ref["tot"], rtol=1e-13, atol=0)
    # the own rows tile the grid
    assert rows[0][0] == 0 and rows[-1][1] == ny
    assert all(rows[k][1] == rows[k + 1][0] for k in range(nslab - 1))


@pytest.mark.parametrize("kind,nslab", [("riemann", 2), ("smooth", 3)])
def test_slab_rhs_bitwise_on_its_own_rows(kind, nslab):
    nx, ny = 40, 72
    lo, hi, bc, x, prim, extra = _case(kind, nx, ny)
    kw = dict(_grid_kw(kind, "fp64"), **extra)
    r = wl.rng(611)
    xdot = r.uniform(-0.2, 0.2, x.shape)
    if bc[1] == esmm.OUTFLOW:
        xdot[:, :, 0] = xdot[:, :, -1] = 0.0
        xdot[:, 0, :] = xdot[:, -1, :] = 0.0
    import oracle
    cfg = oracle.make_cfg(nx, ny, bc=bc, period=(hi[0] - lo[0], hi[1] - lo[1]), p=2, w=5)
    cons, J = oracle.init_state(cfg, prim, x)
    with esmm.Grid((nx, ny), lo, hi, bc=bc, **kw) as g:
        ref_c, ref_J = g.rhs(cons, J, x, np.ascontiguousarray(xdot))
    comm = LocalComm(nslab)
    per = hi[1] - lo[1]
    for s in range(nslab):
        with esmm.Slab((nx, ny), nslab, s, comm.rank(s), lo=lo, hi=hi, bc=bc, **kw) as sl:
            gr = np.arange(sl.ext0, sl.ext1)
            src = gr % ny
            shift = (gr - src) // ny * per
            xs = x[:, src].copy()
            xs[1] += shift[:, None]
            dc, dj = sl.rhs(np.ascontiguousarray(cons[:, src]), np.ascontiguousarray(J[src]),
                            np.ascontiguousarray(xs), np.ascontiguousarray(xdot[:, src]))
            a, b = sl.own0 - sl.ext0, sl.own1 - sl.ext0
            assert np.array_equal(dc[:, a:b], ref_c[:, sl.own0:sl.own1]), s
            assert np.array_equal(dj[a:b], ref_J[sl.own0:sl.own1]), s


def _proc(rank, world, port, out):
    import datetime
    import os

    import torch
    import torch.distributed as dist
    from paper_2107_12027_gb300.comm import TorchComm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        torch.cuda.set_device(0)
        lo, hi, bc, x, prim, extra = _case("riemann", 40, 64)
        with esmm.Slab((40, 64), world, rank, TorchComm(), lo=lo, hi=hi, bc=bc, **dict(_grid_kw("riemann", "fp64"),
                                                                                       **extra)) as g:
            g.state_set(prim, x)
            dts = [g.rk_step() for _ in range(3)]
            out[rank] = (dts, g.own0, g.own1, g.state_get(esmm.GET_CONS), g.totals())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slabs_as_torch_distributed_processes():
    # the multi-rank path: two processes (here on the same GPU, each its own
    # context), slabs exchanging over a gloo group; no kernel of one process
    # waits on the other's, every wait is on the host with a bounded timeout
    import socket

    import torch.multiprocessing as mp
    lo, hi, bc, x, prim, extra = _case("riemann", 40, 64)
    with esmm.Grid((40, 64), lo, hi, bc=bc, **dict(_grid_kw("riemann", "fp64"), **extra)) as g:
        g.state_set(prim, x)
        dts = [g.rk_step() for _ in range(3)]
        cons, tot = g.state_get(esmm.GET_CONS), g.totals()
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_proc, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for r in range(2):
        d, a, b, c, t = res[r]
        assert d == dts
        assert np.array_equal(c, cons[:, a:b])
        assert np.allclose(t, tot, rtol=1e-13, atol=0)


def test_slab_rejects_thin_slabs_and_other_calls():
    comm = LocalComm(2)
    with pytest.raises(esmm.EsmmError):
        esmm.Slab((32, 30), 2, 0, comm.rank(0), bc=(esmm.OUTFLOW, esmm.OUTFLOW))   # 15 rows < the halo
    with esmm.Slab((32, 40), 2, 0, comm.rank(0), bc=(esmm.OUTFLOW, esmm.OUTFLOW)) as sl:
        assert (sl.own0, sl.own1, sl.ext0, sl.ext1) == (0, 20, 0, 36)
        with pytest.raises(esmm.EsmmError):
            sl.mesh_redistribute()
