"""esmm_advance's step graph, through the C ABI on a grid with its own stream:

  * steps replayed from the graph (advance(n), then advance(1) replays of
    the same graph) leave the state, the mesh and the time equal bit for bit
    to the same number of esmm_rk_step calls, in both forms;
  * with profiling on, the graph carries event nodes around the profiled
    kind: every replay adds its launches to the timed count (6 interface
    launches per step), the times are positive, and a change of the mask or
    of the parameters recaptures the graph;
  * a grid on the legacy default stream never captures and still steps.
"""
import numpy as np
import pytest

from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _grid(stream, form):
    return esmm.Grid((72, 64), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5, alpha=1200.0,
                     precision=esmm.MIXED if form == "mixed" else esmm.FP64, stream=stream)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_graph_replays_equal_direct_steps(form):
    import torch
    st = torch.cuda.Stream()
    x = wl.random_mesh(72, 64, wl.rng(901), amp=0.1, lo=(-1, -1), hi=(1, 1), periodic=(False, False))
    prim = wl.quadrant_riemann(x, wl.quadrant_states(wl.rng(902), vmax=0.5), split=(0.1, -0.15))
    out = []
    for mode in ("direct", "graph"):
        with _grid(st.cuda_stream, form) as g:
            g.state_set(prim, x)
            if mode == "direct":
                for _ in range(7):
                    g.rk_step()
            else:
                g.advance(4)          # captures, then four replays
                for _ in range(3):
                    g.advance(1)      # replays of the same graph
            torch.cuda.synchronize()
            out.append((g.state_get(esmm.GET_CONS), g.state_get(esmm.GET_X), g.time()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_profiled_graph_counts_every_replay():
    import torch
    st = torch.cuda.Stream()
    x, prim = wl.riemann_config(64)
    with esmm.Grid((64, 64), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5, alpha=1200.0,
                   stream=st.cuda_stream) as g:
        g.state_set(prim, x)
        g.profile(1 << esmm.KIND_IFACE)
        g.advance(3)
        p = g.profile_read()
        assert p["iface"][2] == 3 * 6 and p["iface"][1] == 3 * 6 and p["iface"][0] > 0.0
        g.profile(1 << esmm.KIND_IFACE)   # same mask: counters cleared, graph kept
        g.advance(1)
        g.advance(1)
        p = g.profile_read()
        assert p["iface"][2] == 2 * 6 and p["iface"][0] > 0.0
        # another mask: the next multi-step call recaptures with its events
        g.profile((1 << esmm.KIND_IFACE) | (1 << esmm.KIND_NODE))
        g.advance(2)
        p = g.profile_read()
        assert p["iface"][2] == 2 * 6
        assert p["node"][2] > 0 and p["node"][2] == p["node"][1] and p["node"][0] > 0.0
        # a parameter change drops the graph: a single step runs directly
        g.set_params(cfl=0.3)
        g.advance(1)
        p = g.profile_read()
        assert p["iface"][2] == 3 * 6


def test_default_stream_grid_steps_without_a_graph():
    x, prim = wl.riemann_config(48)
    with esmm.Grid((48, 48), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5) as g:
        g.state_set(prim, x)
        g.advance(3)
        c = g.state_get(esmm.GET_CONS)
    with esmm.Grid((48, 48), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5) as g:
        g.state_set(prim, x)
        for _ in range(3):
            g.rk_step()
        assert np.array_equal(c, g.state_get(esmm.GET_CONS))
