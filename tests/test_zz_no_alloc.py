"""The allocation-free right-hand side (esmm_rhs_static) against esmm_rhs.

esmm_rhs_static serves callers that cannot allocate device memory, such as
code running under an allocator or a memory budget it does not own: it keeps
its scratch in a file-scope device array instead of a grid's buffers.  This
file is collected last on purpose.  It checks, through the C ABI and on two
calls in a row (the second reusing the scratch the first left behind), that
its output matches the grid-based entry point's for every order p, WENO
order w and with or without a mesh velocity; that the second call leaves the
device's free memory unchanged; and that it rejects sizes beyond its fixed
maximum.
"""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _case(kind, nx, ny, p, w):
    if kind == "smooth":
        x = wl.wavy_mesh(nx, ny, amp=0.04)
        xdot = wl.wavy_mesh_velocity(nx, ny, amp=0.04, t=0.7)
        prim = wl.smooth_random_state(x, wl.rng(91))
        bc, lo, hi = (0, 0), (0.0, 0.0), (1.0, 1.0)
    else:
        x = wl.random_mesh(nx, ny, wl.rng(92), amp=0.2, lo=(-1, -1), hi=(1, 1), periodic=(False, False))
        xdot = wl.rng(93).uniform(-0.3, 0.3, x.shape)
        xdot[:, :, 0] = xdot[:, :, -1] = 0.0
        xdot[:, 0, :] = xdot[:, -1, :] = 0.0
        prim = wl.quadrant_riemann(x, wl.quadrant_states(wl.rng(94)), split=(0.1, -0.2))
        bc, lo, hi = (1, 1), (-1.0, -1.0), (1.0, 1.0)
    cfg = oracle.make_cfg(nx, ny, bc=bc, period=(hi[0] - lo[0], hi[1] - lo[1]), p=p, w=w)
    cons, J = oracle.init_state(cfg, prim, x)
    return bc, lo, hi, cons, J, x, np.ascontiguousarray(xdot)


CASES = [("smooth", (53, 37), 2, 5, True), ("riemann", (61, 45), 2, 5, True),
         ("smooth", (29, 33), 1, 0, True), ("smooth", (31, 27), 3, 3, False),
         ("riemann", (37, 41), 3, 5, False), ("riemann", (33, 29), 1, 3, True)]


@pytest.mark.parametrize("kind,shape,p,w,moving", CASES)
def test_static_rhs_matches_grid_rhs_on_two_calls(kind, shape, p, w, moving):
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    dev = torch.device("cuda", 0)
    nx, ny = shape
    bc, lo, hi, cons, J, x, xdot = _case(kind, nx, ny, p, w)
    if not moving:
        xdot = None
    with esmm.Grid((nx, ny), lo, hi, bc=bc, p=p, w=w) as g:
        ref_c, ref_J = g.rhs(cons, J, x, xdot)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ins = [t(cons), t(J), t(x), t(xdot)]
    dc = torch.empty((4, ny, nx), dtype=torch.float64, device=dev)
    dj = torch.empty((ny, nx), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    free = []
    for call in range(2):
        dc.fill_(np.nan)
        dj.fill_(np.nan)
        rc = esmm.rhs_static(nx, ny, bc, lo, hi, 5.0 / 3.0, p, w, *ins, dc, dj)
        assert rc == esmm.OK
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert _rel(dc.cpu().numpy(), ref_c) < TOL, (kind, call)
        assert _rel(dj.cpu().numpy(), ref_J) < TOL, (kind, call)
    # the second call allocated nothing on the device
    assert free[1] == free[0], free


def test_static_rhs_rejects_oversized_grid():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    n = 300                                  # (300+6)^2 > ESMM_STATIC_MAX_PADDED_NODES
    assert (n + 6) ** 2 > esmm.STATIC_MAX_PADDED_NODES
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device=dev)
    rc = esmm.rhs_static(n, n, (0, 0), (0, 0), (1, 1), 5.0 / 3.0, 2, 5, z(4, n, n), z(n, n), z(2, n, n), None,
                         z(4, n, n), z(n, n))
    assert rc == esmm.ERR_ARG
