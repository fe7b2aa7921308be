"""The fused sweep kernel (pair fluxes kept in shared memory) against the
pair + interface kernels, through the C ABI.

Both variants run the same flux arithmetic in the same order, so they must
agree bit for bit:
  * the right-hand side for every (p, w) in both forms, on grids whose sides
    leave ragged segments (33 - p interfaces per warp and line) and ragged
    line groups, periodic and outflow, on a random curvilinear mesh with a
    mesh velocity;
  * three SSP-RK3 steps with the adaptive mesh and the eq. cfl step;
  * a tuned batch (the tuner picks the variant per direction) against an
    untuned split one.
The parity tests against the oracle run through the default variant (the
fused kernel until a tuner decides), so the two together cover both paths.
"""
import numpy as np
import pytest

from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _case(nx, ny, periodic, seed):
    if periodic:
        lo, hi, bc = (0.0, 0.0), (1.0, 1.0), (esmm.PERIODIC, esmm.PERIODIC)
        x = wl.wavy_mesh(nx, ny, amp=0.04)
        prim = wl.smooth_random_state(x, wl.rng(seed))
    else:
        lo, hi, bc = (-1.0, -1.0), (1.0, 1.0), (esmm.OUTFLOW, esmm.OUTFLOW)
        x = wl.random_mesh(nx, ny, wl.rng(seed), amp=0.15, lo=lo, hi=hi, periodic=(False, False))
        prim = wl.quadrant_riemann(x, wl.quadrant_states(wl.rng(seed + 1), vmax=0.5), split=(0.1, -0.15))
    return lo, hi, bc, x, prim


@pytest.mark.parametrize("form", ["fp64", "mixed"])
@pytest.mark.parametrize("p,w", [(1, 0), (1, 3), (1, 5), (2, 0), (2, 3), (2, 5), (3, 0), (3, 3), (3, 5)])
def test_fused_rhs_equals_split(p, w, form):
    prec = esmm.MIXED if form == "mixed" else esmm.FP64
    for nx, ny, periodic in ((37, 29, False), (70, 33, True)):
        lo, hi, bc, x, prim = _case(nx, ny, periodic, 800 + p + w)
        r = wl.rng(810)
        xdot = r.uniform(-0.2, 0.2, x.shape)
        if not periodic:
            xdot[:, :, 0] = xdot[:, :, -1] = 0.0
            xdot[:, 0, :] = xdot[:, -1, :] = 0.0
        xdot = np.ascontiguousarray(xdot)
        out = []
        for sweep in (esmm.SWEEP_FUSED, esmm.SWEEP_SPLIT):
            with esmm.Grid((nx, ny), lo, hi, bc=bc, p=p, w=w, precision=prec, sweep=sweep) as g:
                g.state_set(prim, x)
                cons, J = g.state_get(esmm.GET_CONS), g.state_get(esmm.GET_J)
                out.append(g.rhs(cons, J, x, xdot))
        assert np.array_equal(out[0][0], out[1][0]), (nx, ny)
        assert np.array_equal(out[0][1], out[1][1]), (nx, ny)
        assert np.isfinite(out[0][0]).all()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_fused_steps_equal_split(form):
    prec = esmm.MIXED if form == "mixed" else esmm.FP64
    lo, hi, bc, x, prim = _case(90, 67, False, 820)
    res = []
    for sweep in (esmm.SWEEP_FUSED, esmm.SWEEP_SPLIT):
        with esmm.Grid((90, 67), lo, hi, bc=bc, p=2, w=5, alpha=1200.0, precision=prec, sweep=sweep) as g:
            assert g.get_params()["sweep"] == sweep
            g.state_set(prim, x)
            dts = [g.rk_step() for _ in range(3)]
            res.append((dts, g.state_get(esmm.GET_CONS), g.state_get(esmm.GET_X)))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][2], res[1][2])


def test_tuned_batch_equals_split_batch():
    sizes = [(40, 40), (64, 48), (33, 70), (96, 96)]
    probs = []
    for k, (nx, ny) in enumerate(sizes):
        lo, hi, bc, x, prim = _case(nx, ny, False, 830 + k)
        probs.append((x, prim))
    res = []
    for tuned in (True, False):
        kw = dict(p=2, w=5, precision=esmm.MIXED, alpha=1200.0)
        if not tuned:
            kw["sweep"] = esmm.SWEEP_SPLIT
        with esmm.Batch(sizes, lo=(-1, -1), hi=(1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), **kw) as b:
            for k, (x, prim) in enumerate(probs):
                b.state_set(k, prim, x)
            if tuned:
                shapes = b.tune()
                assert all(s in (-1, 999) or (s % 1000 in (0, 8, 16, 32, 64, 128) and s // 1000 in (0, 1))
                           for s in shapes[15:17])
            b.advance(3)
            res.append([b.state_get(k, esmm.GET_CONS) for k in range(len(sizes))])
    for a, c in zip(*res):
        assert np.array_equal(a, c)


def test_sweep_parameter_is_checked():
    with esmm.Grid((32, 32)) as g:
        assert g.get_params()["sweep"] == esmm.SWEEP_AUTO
        with pytest.raises(esmm.EsmmError):
            g.set_params(sweep=7)
