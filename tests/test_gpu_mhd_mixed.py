"""Mixed-precision form of the RMHD path (FP32 two-point fluxes, eigen-system,
WENO and dissipation; FP64 recovery, near-equal log means, metric averages,
state and totals) against the FP64 oracle and the FP64 form.

Bounds, relative to each component's max-norm: the EC right-hand side (w = 0)
within 2e-5 -- a difference of interface fluxes some 25x larger, each
rounded to FP32 (eps 6e-8); the ES right-hand side within 5e-3 -- its
dissipation goes through the FP32 Cholesky factor and Jacobi rotations of the
6 x 6 symmetrized pencil, whose eigenvectors carry ~eps/gap error (measured
up to 1.4e-3 at p = 3 on smooth states).  After two rotor steps at 128^2 with
the FP64 form's time steps, the L1 density difference and the total-entropy
difference stay below 1e-4; a constant state on a random mesh stays within
1e-5 for five steps."""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
G43 = 4.0 / 3.0


def _rel_comp(a, b):
    return max(np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() for c in range(a.shape[0]) if np.abs(b[c]).max() > 0)


@pytest.mark.parametrize("p,w,tol", [(2, 5, 5e-3), (3, 5, 5e-3), (2, 0, 2e-5)])
def test_mixed_rmhd_rhs_close_to_oracle(p, w, tol):
    nx, ny = 45, 37
    x = wl.wavy_mesh(nx, ny, amp=0.04)
    xd = wl.wavy_mesh_velocity(nx, ny, amp=0.04, t=1.3)
    prim = wl.smooth_random_state_mhd(x, wl.rng(140 + p + w))
    cfg = oracle.make_cfg(nx, ny, bc=(0, 0), period=(1, 1), p=p, w=w, gamma=G43, phys=oracle.RMHD)
    cons, J = oracle.init_state(cfg, prim, x)
    ref = oracle.rhs(cfg, cons, J, x, xd)
    with esmm.Grid((nx, ny), p=p, w=w, gamma=G43, phys=esmm.RMHD, precision=esmm.MIXED) as g:
        got = g.rhs(cons, J, x, xd)
    assert _rel_comp(got[0], ref[0]) < tol
    assert np.abs(got[1] - ref[1]).max() < 1e-5 * np.abs(ref[1]).max()


def test_mixed_rmhd_discontinuous_and_rotor_rhs():
    nx, ny = 40, 36
    x = wl.random_mesh(nx, ny, wl.rng(160), amp=0.2, lo=(-1, -1), hi=(1, 1), periodic=(False, False))
    prim = wl.quadrant_riemann_mhd(x, wl.quadrant_states_mhd(wl.rng(162)), split=(0.1, -0.2))
    cfg = oracle.make_cfg(nx, ny, bc=(1, 1), period=(2, 2), p=2, w=5, gamma=G43, phys=oracle.RMHD)
    cons, J = oracle.init_state(cfg, prim, x)
    ref = oracle.rhs(cfg, cons, J, x)
    with esmm.Grid((nx, ny), (-1, -1), (1, 1), bc=(1, 1), p=2, w=5, gamma=G43, phys=esmm.RMHD,
                   precision=esmm.MIXED) as g:
        got = g.rhs(cons, J, x)
    assert _rel_comp(got[0], ref[0]) < 5e-3
    n = 64
    x, prim = wl.rotor_config(n)
    cfg = oracle.make_cfg(n, n, bc=(1, 1), period=(1, 1), p=2, w=5, gamma=G43, phys=oracle.RMHD)
    cons, J = oracle.init_state(cfg, prim, x)
    ref = oracle.rhs(cfg, cons, J, x)
    with esmm.Grid((n, n), (-0.5, -0.5), (0.5, 0.5), bc=(1, 1), p=2, w=5, gamma=G43, phys=esmm.RMHD,
                   precision=esmm.MIXED) as g:
        got = g.rhs(cons, J, x)
    assert _rel_comp(got[0], ref[0]) < 5e-3


def test_mixed_rmhd_rotor_error_and_entropy():
    n = 128
    x, prim = wl.rotor_config(n)
    res = {}
    for prec in (esmm.FP64, esmm.MIXED):
        with esmm.Grid((n, n), (-0.5, -0.5), (0.5, 0.5), bc=(1, 1), p=2, w=5, gamma=G43, phys=esmm.RMHD,
                       alpha=800.0, monitor=esmm.MONITOR_LNRHO, precision=prec) as g:
            g.state_set(prim, x)
            if prec == esmm.FP64:
                dts = [g.rk_step() for _ in range(2)]
            else:
                for dt in dts:
                    g.advance(1, dt)
            res[prec] = (g.state_get(esmm.GET_PRIM)[0], g.totals()[0])
    rf, rm = res[esmm.FP64][0], res[esmm.MIXED][0]
    assert np.abs(rm - rf).mean() / np.abs(rf).mean() < 1e-4
    assert abs(res[esmm.MIXED][1] - res[esmm.FP64][1]) < 1e-4 * abs(res[esmm.FP64][1])


def test_mixed_rmhd_free_stream():
    n = 40
    x = wl.random_mesh(n, n, wl.rng(102), amp=0.3)
    w0 = np.array([1.3, 0.3, -0.2, 0.1, 0.7, 0.5, -0.8, 0.3])
    prim = np.ascontiguousarray(np.broadcast_to(w0[:, None, None], (8, n, n)))
    with esmm.Grid((n, n), p=2, w=5, gamma=G43, phys=esmm.RMHD, precision=esmm.MIXED) as g:
        g.state_set(prim, x)
        for _ in range(5):
            g.rk_step()
        got = g.state_get(esmm.GET_PRIM)
    np.testing.assert_allclose(got, prim, rtol=0, atol=1e-5)
