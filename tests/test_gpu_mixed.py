"""Mixed-precision form (FP32 fluxes/WENO/metric averages, FP64 recovery,
near-equal log means, state and totals) against the FP64 oracle and the FP64
form.  Bounds: single right-hand side within 1e-3 of the oracle's max-norm
per component (the right-hand side is a difference of interface fluxes ~25x
larger, each rounded to FP32); after 20 SSP-RK3 steps of a seeded four-quadrant
problem an L1 density error below 1e-4 and a total-entropy difference below
1e-5 relative to the FP64 form; free stream kept to 1e-5."""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.abs(np.asarray(a) - b).max() / np.abs(b).max()


@pytest.mark.parametrize("p,w", [(2, 5), (3, 5), (2, 0)])
def test_mixed_rhs_close_to_oracle(p, w):
    nx, ny = 64, 48
    x = wl.wavy_mesh(nx, ny, amp=0.04)
    xdot = wl.wavy_mesh_velocity(nx, ny, amp=0.04, t=1.1)
    prim = wl.smooth_random_state(x, wl.rng(101))
    cfg = oracle.make_cfg(nx, ny, p=p, w=w)
    cons, J = oracle.init_state(cfg, prim, x)
    ref = oracle.rhs(cfg, cons, J, x, xdot)
    with esmm.Grid((nx, ny), p=p, w=w, precision=esmm.MIXED) as g:
        got = g.rhs(cons, J, x, xdot)
    for a in range(4):
        assert _rel(got[0][a], ref[0][a]) < 1e-3, a
    assert _rel(got[1], ref[1]) < 1e-5


def test_mixed_run_error_and_entropy_drift():
    n = 96
    x, prim = wl.riemann_config(n)
    res = {}
    for prec in (esmm.FP64, esmm.MIXED):
        with esmm.Grid((n, n), (-1, -1), (1, 1), bc=(1, 1), p=2, w=5, alpha=1200.0,
                       monitor=esmm.MONITOR_LNRHO, precision=prec) as g:
            g.state_set(prim, x)
            if prec == esmm.FP64:
                dt = 0.9 * g.cfl_dt()
            g.advance(20, dt)
            res[prec] = (g.state_get(esmm.GET_PRIM)[0], g.totals()[0])
    rf, rm = res[esmm.FP64][0], res[esmm.MIXED][0]
    l1 = np.abs(rm - rf).mean() / np.abs(rf).mean()
    ds = abs(res[esmm.MIXED][1] - res[esmm.FP64][1]) / abs(res[esmm.FP64][1])
    assert l1 < 1e-4, l1
    assert ds < 1e-5, ds


def test_mixed_free_stream():
    n = 40
    x = wl.random_mesh(n, n, wl.rng(102), amp=0.3)
    w0 = np.array([0.7, 0.4, -0.5, 1.3])
    prim = np.ascontiguousarray(np.broadcast_to(w0[:, None, None], (4, n, n)))
    with esmm.Grid((n, n), p=2, w=5, precision=esmm.MIXED) as g:
        g.state_set(prim, x)
        for _ in range(5):
            g.rk_step()
        got = g.state_get(esmm.GET_PRIM)
    np.testing.assert_allclose(got, prim, rtol=1e-5, atol=1e-5)
