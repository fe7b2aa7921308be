"""The RMHD isentropic vortex examples of Sec. 6 on the GPU (sm_103a), through
the C ABI: the monitor with the Laplacian term (element-wise parity of the
mesh velocity with the oracle), the step with the examples' prescribed mesh
motion (esmm_rk_step_given, parity with the oracle's step), and the orders of
accuracy of MM-O6 (p = 3, EC, prescribed mesh, dt ~ h^2) and MM-O5 (p = 3,
w = 5, adaptive mesh with the Laplacian monitor, dt ~ h^(5/3)) against the
exact solution, in 2D and 3D.

Tolerances: EC parity 1e-12 and ES parity 1e-10 (3D: 1e-9) relative per
component, as for the other RMHD parity tests; the mesh velocity 1e-11 as for the other
mesh parity tests.  The orders are measured on grids the oracle would need
minutes to hours for, so there the exact solution is the reference."""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0
TOL = 1e-12
ES_TOL = 1e-10
VORTEX_MONITOR = dict(monitor=esmm.MONITOR_RHO, alpha=20.0, alpha_lap=10.0)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.ndim >= 3 and a.shape[0] in (2, 3, 8):
        top = np.abs(b).max()
        return max(np.abs(a[c] - b[c]).max() / max(np.abs(b[c]).max(), 1e-8 * top, 1e-300)
                   for c in range(a.shape[0]))
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _pair2(n, R, p, w, **kw):
    cfg = oracle.make_cfg(n, n, period=(2 * R, 2 * R), p=p, w=w, gamma=G53, phys=oracle.RMHD, **kw)
    g = esmm.Grid((n, n), (-R, -R), (R, R), p=p, w=w, gamma=G53, phys=esmm.RMHD, **kw)
    return cfg, g


def _pair3(n, R, p, w, **kw):
    m = (n, n, 5 * n)
    cfg = oracle.make_cfg3(*m, period=(2 * R, 2 * R, 10 * R), p=p, w=w, gamma=G53, **kw)
    g = esmm.Grid3(m, (-R, -R, -5 * R), (R, R, 5 * R), p=p, w=w, gamma=G53, **kw)
    return cfg, g


# ------------------------------------------------------------ monitor parity
@pytest.mark.parametrize("alpha_lap", [0.0, 10.0])
def test_laplacian_monitor_mesh_parity_2d(alpha_lap):
    n, R = 40, 5.0
    x = wl.vortex_mesh(n, 0.3, R=R)
    kw = dict(VORTEX_MONITOR, alpha_lap=alpha_lap)
    cfg, g = _pair2(n, R, 3, 5, **kw)
    prim = wl.rmhd_vortex(x, 0.3, R=R)
    cons, J = oracle.init_state(cfg, prim, x)
    xd_ref, tau_ref, dt_ref = oracle.mesh(cfg, cons, J, x)
    with g:
        g.state_set(prim, x)
        xd, tau, dt = g.mesh_redistribute(0.0)
    assert abs(tau - tau_ref) <= 1e-13 * tau_ref
    assert abs(dt - dt_ref) <= 1e-13 * dt_ref
    assert _rel(xd, xd_ref) < 1e-11


def test_laplacian_monitor_mesh_parity_rhd_riemann():
    # the RHD path shares the monitor kernels: the Riemann problem, ln rho
    n = 48
    x, prim = wl.riemann_config(n)
    kw = dict(monitor=esmm.MONITOR_LNRHO, alpha=300.0, alpha_lap=50.0)
    cfg = oracle.make_cfg(n, n, bc=(1, 1), period=(2, 2), p=2, w=5, **kw)
    cons, J = oracle.init_state(cfg, prim, x)
    xd_ref, tau_ref, dt_ref = oracle.mesh(cfg, cons, J, x)
    with esmm.Grid((n, n), (-1, -1), (1, 1), bc=(1, 1), p=2, w=5, **kw) as g:
        g.state_set(prim, x)
        xd, tau, dt = g.mesh_redistribute(0.0)
    assert abs(tau - tau_ref) <= 1e-13 * tau_ref
    assert abs(dt - dt_ref) <= 1e-13 * dt_ref
    assert _rel(xd, xd_ref) < 1e-11


def test_laplacian_monitor_mesh_parity_3d():
    n, R = 6, 5.0
    x = wl.vortex_mesh3(n, 0.3, R=R)
    cfg, g = _pair3(n, R, 3, 5, **VORTEX_MONITOR)
    prim = wl.rmhd_vortex3(x, 0.3, R=R)
    cons, J = oracle.init_state3(cfg, prim, x)
    xd_ref, tau_ref, dt_ref = oracle.mesh3(cfg, cons, J, x)
    with g:
        g.state_set(prim, x)
        xd, tau, dt = g.mesh_redistribute(0.0)
    assert abs(tau - tau_ref) <= 1e-13 * tau_ref
    # the step is the root of eq. cfl with the mesh velocity in the radius;
    # where the displacement term dominates the radius the root amplifies the
    # rounding of the per-node terms (~4e-13 here)
    assert abs(dt - dt_ref) <= 1e-12 * dt_ref
    assert _rel(xd, xd_ref) < 1e-11


# ------------------------------------------------- prescribed-mesh step parity
@pytest.mark.parametrize("p,w,device", [(3, 0, False), (3, 5, False), (2, 5, True)])
def test_rk_step_given_parity_2d(p, w, device):
    import torch
    n, R, dt = 36, 5.0, 0.05
    x = wl.vortex_mesh(n, 0.0, R=R)
    cfg, g = _pair2(n, R, p, w)
    prim = wl.rmhd_vortex(x, 0.0, R=R)
    cons, J = oracle.init_state(cfg, prim, x)
    with g:
        g.state_set(prim, x)
        for s in range(3):
            xd = wl.vortex_mesh_velocity(n, s * dt, R=R)
            cons, J, x = oracle.rk_step_given(cfg, cons, J, x, xd, dt)
            g.rk_step_given(torch.from_numpy(xd).cuda() if device else xd, dt)
        assert abs(g.time() - 3 * dt) < 1e-14
        tol = TOL if w == 0 else ES_TOL
        assert _rel(g.state_get(esmm.GET_CONS), cons) < tol
        assert _rel(g.state_get(esmm.GET_J), J) < TOL
        assert _rel(g.state_get(esmm.GET_X), x) < TOL


@pytest.mark.parametrize("p,w", [(3, 0), (2, 5)])
def test_rk_step_given_parity_3d(p, w):
    n, R, dt = 6, 5.0, 0.05
    x = wl.vortex_mesh3(n, 0.0, R=R)
    cfg, g = _pair3(n, R, p, w)
    prim = wl.rmhd_vortex3(x, 0.0, R=R)
    cons, J = oracle.init_state3(cfg, prim, x)
    with g:
        g.state_set(prim, x)
        for s in range(2):
            xd = wl.vortex_mesh3_velocity(n, s * dt, R=R)
            cons, J, x = oracle.rk_step3_given(cfg, cons, J, x, xd, dt)
            g.rk_step_given(xd, dt)
        # the 3D parity tests' ES tolerance: the 3D frame adds its angle's
        # rounding to the eigenvectors' eps/gap
        tol = TOL if w == 0 else 1e-9
        assert _rel(g.state_get(esmm.GET_CONS), cons) < tol
        assert _rel(g.state_get(esmm.GET_J), J) < TOL
        assert _rel(g.state_get(esmm.GET_X), x) < TOL


def test_named_schemes():
    for name, mm in {"MM-O6": 1, "MM-O5": 1, "UM-O5": 0, "UM-O6": 0}.items():
        with esmm.Grid((8, 8), scheme=name) as g:
            assert g.get_params()["move_mesh"] == mm
    with esmm.Grid((8, 8), scheme="MM-O5", move_mesh=0) as g:      # the caller's switch wins
        assert g.get_params()["move_mesh"] == 0


def test_rk_step_given_rejects_bad_arguments():
    n, R = 16, 5.0
    x = wl.vortex_mesh(n, 0.0, R=R)
    with esmm.Grid((n, n), (-R, -R), (R, R), gamma=G53, phys=esmm.RMHD) as g:
        with pytest.raises(esmm.EsmmError):
            g.rk_step_given(np.zeros((2, n, n)), 0.01)       # no state yet
        g.state_set(wl.rmhd_vortex(x, 0.0, R=R), x)
        with pytest.raises(esmm.EsmmError):
            g.rk_step_given(np.zeros((2, n, n)), 0.0)        # dt must be > 0
        g.rk_step_given(np.zeros((2, n, n)), 0.01)
        assert abs(g.time() - 0.01) < 1e-15


# ------------------------------------------------------- orders of accuracy
def _run_vortex(dim, n, T, scheme, c):
    """rho errors (max, mean) against the exact vortex after time T on an
    n^2 (2D) or n x n x 5n (3D) grid, R = 5: MM-O6 = p 3, EC, the prescribed
    mesh, nst = ceil(T / (c h^2)) steps; MM-O5 = p 3, w 5, the adaptive mesh
    with the Laplacian monitor, steps of c h^(5/3) (so that the spatial
    error dominates, as in the examples); h = 2R/n."""
    import math
    R = 5.0
    h = 2 * R / n
    o6 = scheme == "MM-O6"
    nst = max(4, math.ceil(T / (c * h ** (2.0 if o6 else 5.0 / 3.0))))
    dt = T / nst
    # MM-O6 here steps with the prescribed mesh velocity, so its adaptive
    # redistribution is off; MM-O5 is the named scheme as it stands
    kw = dict(VORTEX_MONITOR, move_mesh=0) if o6 else dict(VORTEX_MONITOR)
    if dim == 2:
        g = esmm.Grid((n, n), (-R, -R), (R, R), scheme=scheme, gamma=G53, phys=esmm.RMHD, **kw)
        x = wl.vortex_mesh(n, 0.0, R=R) if o6 else wl.uniform_mesh(n, n, (-R, -R), (R, R))
        exact, vel = wl.rmhd_vortex, wl.vortex_mesh_velocity
    else:
        m = (n, n, 5 * n)
        g = esmm.Grid3(m, (-R, -R, -5 * R), (R, R, 5 * R), scheme=scheme, gamma=G53, **kw)
        x = wl.vortex_mesh3(n, 0.0, R=R) if o6 else wl.uniform_mesh3(m, (-R, -R, -5 * R), (R, R, 5 * R))
        exact, vel = wl.rmhd_vortex3, wl.vortex_mesh3_velocity
    with g:
        g.state_set(exact(x, 0.0, R=R), x)
        for s in range(nst):
            if o6:
                g.rk_step_given(vel(n, s * dt, R=R), dt)
            else:
                g.rk_step(dt, sync=False)
        t = g.time()
        xf, rho = g.state_get(esmm.GET_X), g.state_get(esmm.GET_PRIM)[0]
    assert abs(t - T) < 1e-12
    d = np.abs(rho - exact(xf, t, R=R)[0])
    return d.max(), d.mean()


@pytest.mark.parametrize("dim,n,T,scheme,c,omax,o1", [
    (2, 80, 4.0, "MM-O6", 0.2, 5.2, 5.5),
    (2, 80, 4.0, "MM-O5", 0.1, 2.9, 4.0),
    (3, 32, 0.1, "MM-O6", 0.2, 4.5, 4.8),
    (3, 32, 0.1, "MM-O5", 0.1, 2.6, 3.0),
])
def test_vortex_order(dim, n, T, scheme, c, omax, o1):
    # The examples' convergence study (Sec. 6; t = 4 in 2D, t = 0.1 in 3D)
    # between n and 2n.  Measured on GB300: 2D MM-O6 orders 5.6 (max) and 5.8
    # (mean), MM-O5 3.2 and 4.4, 3D MM-O6 4.8 and 5.1, MM-O5 2.9 and 3.4.
    # MM-O5's orders at these sizes are pre-asymptotic: the WENO epsilon
    # (1e-6, 1e-12, h^2) and the mesh (static, prescribed, adaptive) leave
    # them unchanged, and on a static mesh they rise to 4.6 between 160 and
    # 320 nodes per side.
    e1, e2 = _run_vortex(dim, n, T, scheme, c), _run_vortex(dim, 2 * n, T, scheme, c)
    assert np.log2(e1[0] / e2[0]) > omax, (e1, e2)
    assert np.log2(e1[1] / e2[1]) > o1, (e1, e2)


def test_vortex_entropy_ec_and_es_on_gpu():
    # total entropy sum J eta (Thm. 3.1 / 4.1): MM-O6 changes it only by the
    # RK3 error, which falls ~8x per halving of dt; MM-O5 on the adaptive mesh
    # decreases it in every step
    n, R, T = 48, 5.0, 0.5
    x0 = wl.vortex_mesh(n, 0.0, R=R)
    dS = []
    for nst in (10, 20):
        dt = T / nst
        with esmm.Grid((n, n), (-R, -R), (R, R), p=3, w=0, gamma=G53, phys=esmm.RMHD, move_mesh=0) as g:
            g.state_set(wl.rmhd_vortex(x0, 0.0, R=R), x0)
            s0 = g.totals()[0]
            for s in range(nst):
                g.rk_step_given(wl.vortex_mesh_velocity(n, s * dt, R=R), dt)
            dS.append(g.totals()[0] - s0)
    assert dS[0] / dS[1] > 7.0, dS
    x = wl.uniform_mesh(n, n, (-R, -R), (R, R))
    with esmm.Grid((n, n), (-R, -R), (R, R), p=3, w=5, gamma=G53, phys=esmm.RMHD, **VORTEX_MONITOR) as g:
        g.state_set(wl.rmhd_vortex(x, 0.0, R=R), x)
        S = [g.totals()[0]]
        for s in range(20):
            g.rk_step(0.0)                 # the CFL step of eq. cfl
            S.append(g.totals()[0])
    assert (np.diff(S) < 0).all(), np.diff(S)
