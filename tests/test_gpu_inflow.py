"""The inflow boundary (the shock-cloud examples of Sec. 6) on the GPU against
the oracle, element by element: 2D RHD and RMHD right-hand sides and steps
with an inflow end, the 3D right-hand side, and the calls' error paths.
Tolerances as for the other parity tests of each system: 1e-12 for the EC
scheme and RHD, 1e-10 for the RMHD ES scheme (eigenvectors resolved to
~eps/gap), per component relative to its max-norm.  A component that vanishes
identically (v_2, v_3 and B_1 of the shock-cloud data, whose computed rates
are the rounding noise, ~1e-16, of flux differences of O(1) terms) is
compared at 1e-5 of the largest component instead."""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.ndim >= 3 and a.shape[0] in (4, 8):
        top = np.abs(b).max()
        return max(np.abs(a[c] - b[c]).max() / max(np.abs(b[c]).max(), 1e-5 * top, 1e-300)
                   for c in range(a.shape[0]))
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("p,w", [(2, 5), (3, 0)])
def test_rhd_rhs_parity_with_inflow(p, w):
    nx, ny = 37, 29
    x = wl.random_mesh(nx, ny, wl.rng(700 + p), amp=0.2, lo=(-1, -1), hi=(1, 1), periodic=(False, False))
    xdot = wl.rng(701).uniform(-0.3, 0.3, x.shape)
    xdot[:, :, 0] = xdot[:, :, -1] = xdot[:, 0, :] = xdot[:, -1, :] = 0.0
    xdot = np.ascontiguousarray(xdot)
    prim = wl.quadrant_riemann(x, wl.quadrant_states(wl.rng(702)), split=(0.1, -0.2))
    w_in = (2.0, 0.6, -0.2, 1.5)
    cfg = oracle.make_cfg(nx, ny, bc=(oracle.INFLOW, oracle.OUTFLOW), period=(2, 2), p=p, w=w, inflow=w_in)
    cons, J = oracle.init_state(cfg, prim, x)
    ref = oracle.rhs(cfg, cons, J, x, xdot)
    with esmm.Grid((nx, ny), (-1, -1), (1, 1), bc=(esmm.INFLOW, esmm.OUTFLOW), p=p, w=w) as g:
        g.set_inflow(w_in)
        got = g.rhs(cons, J, x, xdot)
    assert _rel(got[0], ref[0]) < 1e-12
    assert _rel(got[1], ref[1]) < 1e-12


def test_rmhd_shock_cloud_rhs_and_steps_parity():
    n = (42, 30)
    x, prim = wl.rmhd_shock_cloud_config(n)
    # an inflow state off the initial boundary data, so that the ghosts matter
    w_in = np.array(wl.SHOCK_CLOUD_POST) * [1.05, 1.0, 1.0, 1.0, 1.1, 1.0, 1.0, 1.0]
    kw = dict(p=3, w=5)
    cfg = oracle.make_cfg(*n, bc=(oracle.INFLOW, oracle.OUTFLOW), period=(1.4, 1.0), gamma=G53, phys=oracle.RMHD,
                          inflow=w_in, monitor=oracle.MONITOR_LNRHO, alpha=800.0, **kw)
    cons, J = oracle.init_state(cfg, prim, x)
    ref = oracle.rhs(cfg, cons, J, x)
    with esmm.Grid(n, (-0.2, 0.0), (1.2, 1.0), bc=(esmm.INFLOW, esmm.OUTFLOW), gamma=G53, phys=esmm.RMHD,
                   monitor=esmm.MONITOR_LNRHO, alpha=800.0, **kw) as g:
        g.set_inflow(w_in)
        got = g.rhs(cons, J, x)
        assert _rel(got[0], ref[0]) < 1e-10
        assert _rel(got[1], ref[1]) < 1e-12
        # three adaptive-mesh steps
        g.state_set(prim, x)
        c, Jr, xr = cons, J, x
        for _ in range(3):
            dt = g.rk_step()
            c, Jr, xr, = oracle.rk_step(cfg, c, Jr, xr, dt)[:3]
        assert _rel(g.state_get(esmm.GET_CONS), c) < 1e-10
        assert _rel(g.state_get(esmm.GET_X), xr) < 1e-10


def test_rmhd_shock_cloud_3d_rhs_parity():
    n = (14, 10, 10)
    x, prim = wl.rmhd_shock_cloud3_config(n)
    w_in = np.array(wl.SHOCK_CLOUD_POST) * [1.05, 1.0, 1.0, 1.0, 1.1, 1.0, 1.0, 1.0]
    cfg = oracle.make_cfg3(*n, bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.OUTFLOW), period=(1.4, 1.0, 1.0),
                           gamma=G53, p=2, w=5, inflow=w_in)
    cons, J = oracle.init_state3(cfg, prim, x)
    ref = oracle.rhs3(cfg, cons, J, x)
    with esmm.Grid3(n, (-0.2, 0.0, 0.0), (1.2, 1.0, 1.0), bc=(esmm.INFLOW, esmm.OUTFLOW, esmm.OUTFLOW),
                    gamma=G53, p=2, w=5) as g:
        g.set_inflow(w_in)
        got = g.rhs(cons, J, x)
    assert _rel(got[0], ref[0]) < 1e-9
    assert _rel(got[1], ref[1]) < 1e-12


def test_inflow_error_paths():
    n = (16, 12)
    x, prim = wl.rmhd_shock_cloud_config(n)
    with esmm.Grid(n, (-0.2, 0.0), (1.2, 1.0), bc=(esmm.INFLOW, esmm.OUTFLOW), gamma=G53, phys=esmm.RMHD) as g:
        g.state_set(prim, x)
        with pytest.raises(esmm.EsmmError, match="STATE"):
            g.rk_step()                                        # no inflow state yet
        with pytest.raises(esmm.EsmmError, match="ARG"):
            g.set_inflow((1.0, 0.99, 0.5, 0.0, 1.0, 0.0, 0.0, 0.0))   # |v| >= 1
        g.set_inflow(wl.SHOCK_CLOUD_POST)
        g.rk_step()
        with pytest.raises(esmm.EsmmError, match="ARG"):
            g.adjoint_record(1)                                # the adjoint takes periodic/outflow ends


def test_shock_cloud_runs_admissibly():
    # the 2D shock-cloud at the example's 210 x 150 mesh, MM-O5, 40 steps
    n = (210, 150)
    x, prim = wl.rmhd_shock_cloud_config(n)
    with esmm.Grid(n, (-0.2, 0.0), (1.2, 1.0), bc=(esmm.INFLOW, esmm.OUTFLOW), gamma=G53, phys=esmm.RMHD,
                   scheme="MM-O5", monitor=esmm.MONITOR_LNRHO, alpha=800.0) as g:
        g.set_inflow(wl.SHOCK_CLOUD_POST)
        g.state_set(prim, x)
        m0 = g.totals()[1]
        g.advance(40)
        nfail, _ = g.last_error()
        assert nfail == 0 and g.time() > 0
        got = g.state_get(esmm.GET_PRIM)
        assert np.isfinite(got).all() and got[0].min() > 0 and got[4].min() > 0
        # mass enters through the inflow end: the total grows by the inflow flux
        assert g.totals()[1] > m0
