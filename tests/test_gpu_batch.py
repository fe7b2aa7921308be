"""Batched form: independent problems of different sizes in one handle.

Every kernel of a batched step covers all problems in one launch (block ->
(problem, tile) map) and steps are replayed from a CUDA graph.  Each problem
must evolve exactly as it does alone (FP64: 1e-12 relative, the single-grid
path being itself at 1e-12 of the oracle), one problem is also checked
against the oracle directly, and the autotuned launch shapes must not change
the results.
"""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rel(a, b):
    return np.abs(np.asarray(a) - b).max() / np.abs(b).max()


def _problems():
    # (size, bc, lo, hi, mesh, prim)
    out = []
    for k, (nx, ny) in enumerate([(40, 32), (64, 48), (33, 57), (20, 20)]):
        if k % 2 == 0:
            x = wl.uniform_mesh(nx, ny, (-1, -1), (1, 1), (False, False))
            prim = wl.quadrant_riemann(x, wl.quadrant_states(wl.rng(200 + k)))
            out.append(((nx, ny), (1, 1), (-1.0, -1.0), (1.0, 1.0), x, prim))
        else:
            x = wl.wavy_mesh(nx, ny, amp=0.03)
            prim = wl.smooth_random_state(x, wl.rng(210 + k))
            out.append(((nx, ny), (0, 0), (0.0, 0.0), (1.0, 1.0), x, prim))
    return out


def _run_single(prob, steps, precision):
    size, bc, lo, hi, x, prim = prob
    with esmm.Grid(size, lo, hi, bc=bc, p=2, w=5, alpha=200.0, precision=precision) as g:
        g.state_set(prim, x)
        for _ in range(steps):
            g.rk_step()
        return g.state_get(esmm.GET_CONS), g.state_get(esmm.GET_J), g.state_get(esmm.GET_X), g.time()


@pytest.mark.parametrize("precision", [esmm.FP64, esmm.MIXED])
def test_batch_matches_single_problems(precision):
    probs = _problems()
    steps = 4
    with esmm.Batch([p[0] for p in probs], lo=[p[2] for p in probs], hi=[p[3] for p in probs],
                    bc=[p[1] for p in probs], p=2, w=5, alpha=200.0, precision=precision) as b:
        for k, pr in enumerate(probs):
            b.state_set(k, pr[5], pr[4])
        b.advance(steps)                       # graph replays
        t = b.times()
        got = [(b.state_get(k, esmm.GET_CONS), b.state_get(k, esmm.GET_J), b.state_get(k, esmm.GET_X))
               for k in range(len(probs))]
    tol = TOL if precision == esmm.FP64 else 1e-6
    for k, pr in enumerate(probs):
        c, J, x, ts = _run_single(pr, steps, precision)
        assert abs(t[k] / ts - 1) < 1e-13, k
        assert _rel(got[k][0], c) < tol, k
        assert _rel(got[k][1], J) < tol, k
        assert _rel(got[k][2], x) < tol, k


def test_batch_problem_against_oracle_and_tuning_invariance():
    probs = _problems()
    with esmm.Batch([p[0] for p in probs], lo=[p[2] for p in probs], hi=[p[3] for p in probs],
                    bc=[p[1] for p in probs], p=2, w=5, alpha=200.0) as b:
        for k, pr in enumerate(probs):
            b.state_set(k, pr[5], pr[4])
        shapes = b.tune()
        assert len(shapes) == esmm.TUNE_SLOTS
        assert all(abs(s) in (64, 128, 256, 512) for s in shapes[:13])
        # pair slots: a tile shape (+1000: persistent); interface slots also
        # -1 / 999: the fused sweep kernel (+1000: persistent)
        split = lambda s: s % 1000 in (0, 8, 16, 32, 64, 128) and s // 1000 in (0, 1)
        assert all(split(s) for s in shapes[13:15])
        assert all(split(s) or s in (-1, 999) for s in shapes[15:17])
        b.advance(2)
        got = b.state_get(1, esmm.GET_CONS)
        totals = b.totals()
    size, bc, lo, hi, x, prim = probs[1]
    cfg = oracle.make_cfg(size[0], size[1], bc=bc, period=(1.0, 1.0), p=2, w=5, alpha=200.0)
    cons, J = oracle.init_state(cfg, prim, x)
    for _ in range(2):
        cons, J, x, _ = oracle.rk_step(cfg, cons, J, x)
    assert _rel(got, cons) < TOL
    ref_tot = oracle.totals(cfg, cons, J)
    np.testing.assert_allclose(totals[1], ref_tot[:3], rtol=1e-12)


def test_graph_replay_equals_step_by_step():
    x, prim = wl.riemann_config(48)
    res = []
    for use_graph in (False, True):
        with esmm.Batch([(48, 48)], lo=(-1, -1), hi=(1, 1), bc=(1, 1), p=2, w=5, alpha=1200.0) as b:
            b.state_set(0, prim, x)
            if use_graph:
                b.advance(5)
            else:
                for _ in range(5):
                    b.rk_step(sync=False)
            res.append(b.state_get(0, esmm.GET_CONS))
    assert _rel(res[1], res[0]) < 1e-15


@pytest.mark.parametrize("precision", [esmm.FP64, esmm.MIXED])
def test_tile_shapes_and_persistent_grids_change_nothing(precision):
    # each pair and interface is computed by one thread whatever tile holds
    # it and whichever block of a persistent grid takes that tile: a tuned
    # grid (tile shapes, persistence) steps bit for bit as an untuned one
    x, prim = wl.riemann_config(72)
    res = []
    for tuned in (False, True):
        with esmm.Grid((72, 72), (-1, -1), (1, 1), bc=(1, 1), p=2, w=5, alpha=1200.0, precision=precision) as g:
            g.state_set(prim, x)
            if tuned:
                shapes = g.tune()
                assert len(shapes) == esmm.TUNE_SLOTS
            for _ in range(3):
                g.rk_step()
            res.append(g.state_get(esmm.GET_CONS))
    assert np.array_equal(res[0], res[1])
