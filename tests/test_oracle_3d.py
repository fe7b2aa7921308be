"""Pins of the 3D RMHD oracle against what the paper and the mathematics fix:
the discrete SCL of the nested conservative metrics (eq. SCLCoeff, proved
from the commutativity of the central differences), exact metrics on affine
meshes, the EC entropy identity with the Powell source on a moving mesh
(Thm. 3.1), the ES entropy inequality (Thm. 4.1), free-stream preservation
(Prop. 3.2), conservation of mass across periodic seams, the 3D mesh
redistribution (uniform-monitor fixed point, limiter, the step of eq. cfl
with the mesh velocity), and short runs of the 3D blast."""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import workloads as wl

N3 = (7, 6, 5)


def _delta(a, k, p):
    """2p-th order central difference along direction k of a periodic field
    a[z][y][x] (axis 2 - k), written out from delta_k of Sec. 3.3."""
    al = oracle.alpha(p)
    out = np.zeros_like(a)
    for n in range(1, p + 1):
        out += 0.5 * al[n - 1] * (np.roll(a, -n, axis=2 - k) - np.roll(a, n, axis=2 - k))
    return out


@pytest.mark.parametrize("p", [1, 2, 3])
def test_discrete_scl_3d(p):
    c = oracle.make_cfg3(*N3, p=p)
    x = wl.random_mesh3(N3, wl.rng(400 + p), amp=0.2)
    m, _ = oracle.metrics3(c, x)
    M = m.reshape(3, 3, *m.shape[1:])
    for j in range(3):
        s = sum(_delta(M[k, j], k, p) for k in range(3))
        assert np.abs(s).max() < 1e-15 * max(np.abs(M).max(), 1.0) * 100


def test_metrics_exact_on_affine_mesh_3d():
    # x = A xi + b: J d xi_k/d x_j = cof(A)_{jk}, J = det(A)
    c = oracle.make_cfg3(*N3, bc=(1, 1, 1), p=2)
    A = np.array([[0.11, 0.02, -0.01], [0.015, 0.09, 0.02], [-0.01, 0.025, 0.13]])
    k, j, i = np.meshgrid(np.arange(N3[2]), np.arange(N3[1]), np.arange(N3[0]), indexing="ij")
    xi = np.stack([i, j, k]).astype(float)
    x = np.ascontiguousarray(np.einsum("ab,b...->a...", A, xi) + np.array([0.3, -0.2, 0.1])[:, None, None, None])
    m, J0 = oracle.metrics3(c, x)
    cof = np.linalg.det(A) * np.linalg.inv(A)        # cof(A)^T = det(A) A^{-1}
    for kk in range(3):
        for jj in range(3):
            np.testing.assert_allclose(m[3 * kk + jj], cof[kk, jj], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(J0, np.linalg.det(A), rtol=1e-12)


def _smooth3(p, w, seed):
    c = oracle.make_cfg3(*N3, p=p, w=w)
    x = wl.wavy_mesh3(N3, amp=0.04)
    xd = wl.wavy_mesh_velocity3(N3, amp=0.04, t=1.1)
    prim = wl.smooth_random_state_mhd3(x, wl.rng(seed))
    cons, J = oracle.init_state3(c, prim, x)
    return c, cons, J, x, xd


@pytest.mark.parametrize("p", [1, 2, 3])
def test_ec_entropy_identity_3d(p):
    c, cons, J, x, xd = _smooth3(p, 0, 410 + p)
    dc, dJ = oracle.rhs3(c, cons, J, x, xd)
    prod = oracle.totals3(c, cons, J, dc, dJ)[3]
    assert abs(prod) < 1e-14 * np.abs(dc).sum()


def test_es_entropy_inequality_and_conservation_3d():
    # the ES flux of a periodic seam interface is the same from both sides,
    # so the mass telescopes also on a curvilinear mesh (this fails when the
    # tangential frame follows rounding noise at a normal along x_3)
    c, cons, J, x, xd = _smooth3(2, 5, 420)
    dc, dJ = oracle.rhs3(c, cons, J, x, xd)
    assert oracle.totals3(c, cons, J, dc, dJ)[3] < 0.0
    assert abs(dc[0].sum()) < 1e-13 * np.abs(dc[0]).sum()
    assert abs(dJ.sum()) < 1e-13 * max(np.abs(dJ).sum(), 1e-30) + 1e-18


@pytest.mark.parametrize("w", [0, 5])
def test_free_stream_3d(w):
    c = oracle.make_cfg3(*N3, p=2, w=w)
    x = wl.random_mesh3(N3, wl.rng(430), amp=0.15)
    xd = np.ascontiguousarray(wl.random_mesh3(N3, wl.rng(431), amp=0.1) - wl.uniform_mesh3(N3))
    w0 = np.array([1.3, 0.3, -0.2, 0.1, 0.7, 0.5, -0.8, 0.3])
    prim = np.ascontiguousarray(np.broadcast_to(w0[:, None, None, None], (8,) + N3[::-1]))
    cons, J = oracle.init_state3(c, prim, x)
    dc, dJ = oracle.rhs3(c, cons, J, x, xd)
    U0 = oracle.mhd_prim2cons(c.gamma, w0)
    assert np.abs(dc - U0[:, None, None, None] * dJ[None]).max() < 1e-13 * np.abs(U0).max()


def test_rhs_invariant_under_rotation_of_the_problem():
    # rotating the whole problem by 90 degrees about x_3 (x -> y, y -> -x)
    # rotates the right-hand side: the tangential frame follows the state,
    # not the coordinate axes
    n = 6
    c = oracle.make_cfg3(n, n, n, p=2, w=5)
    x = wl.uniform_mesh3((n, n, n))
    prim = wl.smooth_random_state_mhd3(x, wl.rng(440))
    cons, J = oracle.init_state3(c, prim, x)
    dc, _ = oracle.rhs3(c, cons, J, x)

    def rot(a, vec_comps):
        # field rotation: new(i', j') = old at the preimage; (i, j) -> (j', i') = (n-1-i... )
        b = np.rot90(a, k=1, axes=(-1, -2)).copy()    # rotate the index plane
        for (cx, cy) in vec_comps:
            bx, by = b[cx].copy(), b[cy].copy()
            b[cx], b[cy] = -by, bx
        return np.ascontiguousarray(b)

    prim_r = rot(prim, [(1, 2), (5, 6)])
    # the rotated periodic mesh: a uniform mesh again (spacing is isotropic)
    cons_r, J_r = oracle.init_state3(c, prim_r, x)
    dc_r, _ = oracle.rhs3(c, cons_r, J_r, x)
    np.testing.assert_allclose(dc_r, rot(dc, [(1, 2), (5, 6)]), rtol=0, atol=1e-12 * np.abs(dc).max())


def test_mesh_uniform_monitor_and_step_3d():
    m = 10
    c = oracle.make_cfg3(m, m, m, bc=(1, 1, 1), period=(1, 1, 1), p=2, w=5)
    x = wl.uniform_mesh3((m, m, m), (-0.5,) * 3, (0.5,) * 3, (False,) * 3)
    w0 = np.array([1.0, 0.1, 0.0, -0.1, 1.0, 0.2, 0.1, 0.0])
    prim = np.ascontiguousarray(np.broadcast_to(w0[:, None, None, None], (8, m, m, m)))
    cons, J = oracle.init_state3(c, prim, x)
    xd, tau, dt = oracle.mesh3(c, cons, J, x)
    assert np.abs(xd).max() < 1e-11
    assert abs(dt - oracle.cfl_dt3(c, cons, J, x)) <= 1e-12 * dt
    # the blast: the mesh moves, boundary nodes stay, the mesh Courant number
    # is at most CFL/2 and the step shrinks accordingly
    x, prim = wl.blast3_config(m)
    cons, J = oracle.init_state3(c, prim, x)
    xd, tau, dt = oracle.mesh3(c, cons, J, x)
    dts = oracle.cfl_dt3(c, cons, J, x)
    assert np.abs(xd).max() > 0 and 0 < tau <= 1 and dt < dts
    for d in range(3):
        sl = [slice(None)] * 3
        for end in (0, -1):
            sl[2 - d] = end
            assert np.all(xd[(d,) + tuple(sl)] == 0.0)
    mm, _ = oracle.metrics3(c, x)
    cm = sum((np.abs(sum(xd[j] * mm[3 * k + j] for j in range(3))) * dt / J).max() for k in range(3))
    assert cm <= 0.5 * c.cfl * (1 + 1e-12)


def test_blast_steps_3d():
    m = 14
    c = oracle.make_cfg3(m, m, m, bc=(1, 1, 1), period=(1, 1, 1), p=2, w=5, cfl=0.3)
    x, prim = wl.blast3_config(m)
    cons, J = oracle.init_state3(c, prim, x)
    m0 = cons[0].sum()
    for _ in range(2):
        cons, J, x, dt = oracle.rk_step3(c, cons, J, x)
    pr, st = oracle.state_prim3(c, cons, J)
    assert st == 0 and pr[0].min() > 0 and pr[4].min() > 0
    # outflow boundaries: mass changes only by boundary fluxes.  The ghost
    # nodes of an outflow face are re-extrapolated from the moving interior, so
    # they move (at -xdot of their mirror node) and the face carries a small
    # temporal-metric flux even where the gas is at rest.
    assert abs(cons[0].sum() - m0) < 1e-2 * m0


@pytest.mark.parametrize("alpha_lap", [0.0, 10.0])
def test_monitor_closed_form_on_trigonometric_sigma_3d(alpha_lap):
    # sigma = rho = 1 + sum_d a_d cos(t_d i_d) on a periodic grid: central
    # first differences -a_d sin(t_d) sin(t_d i_d), the seven-point Laplacian
    # sum_d 2 a_d (cos t_d - 1) cos(t_d i_d) (sum-to-product identities); with
    # every n_d a multiple of 4 the gradient's maximum is reached at
    # (n/4, n/4, n/4) and the Laplacian's at the origin (the monitor of the 3D
    # vortex example, Sec. 6).
    n, a = (8, 12, 4), (0.1, 0.05, 0.02)
    t = [2 * np.pi / m for m in n]
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = (i, j, k)
    rho = 1.0 + sum(a[d] * np.cos(t[d] * idx[d]) for d in range(3))
    z = 0.0 * rho
    prim = np.ascontiguousarray(np.stack([rho, z + 0.1, z - 0.05, z + 0.02, z + 1.0, z + 0.2, z + 0.1, z - 0.1]))
    x = wl.uniform_mesh3(n)
    c = oracle.make_cfg3(*n, monitor=oracle.MONITOR_RHO, alpha=20.0, alpha_lap=alpha_lap)
    cons, J = oracle.init_state3(c, prim, x)
    g = np.sqrt(sum((a[d] * np.sin(t[d]) * np.sin(t[d] * idx[d])) ** 2 for d in range(3)))
    lap = np.abs(sum(2 * a[d] * (np.cos(t[d]) - 1) * np.cos(t[d] * idx[d]) for d in range(3)))
    gmax = np.sqrt(sum((a[d] * np.sin(t[d])) ** 2 for d in range(3)))
    lmax = sum(2 * a[d] * (1 - np.cos(t[d])) for d in range(3))
    want = np.sqrt(1.0 + 20.0 * g / gmax + alpha_lap * lap / lmax)
    assert np.abs(oracle.monitor3(c, cons, J) - want).max() < 1e-12


def test_inflow_free_stream_3d():
    # the 3D inflow end (the 3D shock-cloud's boundary): the inflow state
    # everywhere on a random moving mesh is a free stream (Prop. 3.2)
    n = (8, 7, 6)
    w_in = np.array([0.7, 0.3, -0.1, 0.2, 1.3, 0.4, -0.2, 0.1])
    x = wl.random_mesh3(n, wl.rng(660), amp=0.2, periodic=(False, False, True))
    xdot = wl.rng(661).uniform(-0.2, 0.2, x.shape)
    xdot[:, :, :, 0] = xdot[:, :, :, -1] = 0.0     # the non-periodic ends' nodes stay
    xdot[:, :, 0, :] = xdot[:, :, -1, :] = 0.0
    c = oracle.make_cfg3(*n, bc=(oracle.INFLOW, oracle.OUTFLOW, oracle.PERIODIC), period=(1.0, 1.0, 1.0),
                         p=2, w=5, inflow=w_in)
    prim = np.ascontiguousarray(np.broadcast_to(w_in[:, None, None, None], (8,) + tuple(x.shape[1:])))
    cons, J = oracle.init_state3(c, prim, x)
    d, dJ = oracle.rhs3(c, cons, J, x, np.ascontiguousarray(xdot))
    U = cons / J
    assert np.abs(d - U * dJ).max() < 1e-12 * max(np.abs(U * dJ).max(), 1e-300)
