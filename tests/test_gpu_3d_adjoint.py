"""3D RMHD adjoint against finite differences.

  * (d rhs/d cons)^T mu from the 3D adjoint kernels against central
    differences of the GPU right-hand side and of the 3D oracle's, in random
    directions, on smooth periodic states on a moving curvilinear mesh.  The
    interface frame of Sec. 4 is turned to the tangential B of the interface
    state, so the derivative also runs through that angle.
  * The gradient of a final-time functional with respect to the initial
    pressure through recorded SSP-RK3 steps (per-step checkpoints) against
    central differences of the oracle's steps with the recorded mesh
    velocities and time steps (EC 1e-6; ES 5e-2 where differences straddle
    flips of the frozen sign switch Y, as in 2D).
  * The blast workload (32^3 and 128^3, 20 steps; J D and J E integrated
    over [0, 0.2]^3): the adjoint's derivative along the initial pressure
    against central differences of the GPU's recorded map, on the blast with
    relative noise 1e-6 (see _noisy_blast).
"""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
G43 = 4.0 / 3.0


@pytest.mark.parametrize("p,w", [(2, 0), (2, 5), (1, 3)])
def test_rhs_vjp_3d_against_finite_differences(p, w):
    n = (9, 8, 7)
    x = wl.wavy_mesh3(n, amp=0.04)
    xd = np.ascontiguousarray(wl.wavy_mesh_velocity3(n, amp=0.04, t=1.2))
    prim = wl.smooth_random_state_mhd3(x, wl.rng(650))
    cfg = oracle.make_cfg3(*n, p=p, w=w)
    cons, J = oracle.init_state3(cfg, prim, x)
    r = wl.rng(651 + p + w)
    mu = r.standard_normal(cons.shape)
    with esmm.Grid3(n, p=p, w=w) as g:
        lam = g.rhs_vjp(cons, J, x, xd, mu)
        for trial in range(3):
            v = r.standard_normal(cons.shape) * (np.abs(cons) + 1e-3 * np.abs(cons).max()) * 1e-2
            eps = 1e-6
            adj = float((lam * v).sum())
            dg = (g.rhs(cons + eps * v, J, x, xd)[0] - g.rhs(cons - eps * v, J, x, xd)[0]) / (2 * eps)
            do = (oracle.rhs3(cfg, cons + eps * v, J, x, xd)[0] - oracle.rhs3(cfg, cons - eps * v, J, x, xd)[0]) / (2 * eps)
            fg, fo = float((mu * dg).sum()), float((mu * do).sum())
            assert abs(adj - fg) <= 1e-5 * abs(fg), (trial, adj, fg)
            assert abs(adj - fo) <= 1e-5 * abs(fo), (trial, adj, fo)


def _box_weights(x, lo, hi):
    wts = np.zeros((8,) + x.shape[1:])
    inside = np.ones(x.shape[1:], dtype=bool)
    for d in range(3):
        inside &= (x[d] >= lo) & (x[d] <= hi)
    wts[0][inside] = 1.0
    return wts, inside


@pytest.mark.parametrize("w,tol", [(0, 1e-6), (5, 5e-2)])
def test_multistep_adjoint_3d_against_oracle_fd(w, tol):
    steps, m = 2, 8
    x = wl.uniform_mesh3((m, m, m))
    prim = wl.smooth_random_state_mhd3(x, wl.rng(660))
    with esmm.Grid3((m, m, m), p=2, w=w, alpha=200.0) as g:
        g.state_set(prim, x)
        g.adjoint_record(steps)
        dts = g.adjoint_steps()
        xdots = [g.adjoint_checkpoint(k, esmm.GET_XDOT) for k in range(steps)]
        assert np.abs(xdots[0]).max() > 0.0
        wts, _ = _box_weights(g.state_get(esmm.GET_X), 0.0, 0.4)
        wts[4] = wts[0]                           # J D + J E over the box
        _, lam_prim = g.adjoint_vjp(wts)
        cfg = oracle.make_cfg3(m, m, m, p=2, w=w, alpha=200.0)

        def F_oracle(pr):
            cons, J = oracle.init_state3(cfg, pr, x)
            xs = x
            for k in range(steps):
                cons, J, xs = oracle.rk_step3_given(cfg, cons, J, xs, xdots[k], dts[k])
            return float((wts * cons).sum())

        def F_gpu(pr):
            g.state_set(pr, x)
            g.adjoint_replay(steps)
            return float((wts * g.state_get(esmm.GET_CONS)).sum())

        r = wl.rng(661)
        for trial in range(2):
            v = np.zeros_like(prim)
            v[4] = r.standard_normal(prim.shape[1:]) * prim[4]
            eps = 1e-6
            adj = float((lam_prim * v).sum())
            fd_o = (F_oracle(prim + eps * v) - F_oracle(prim - eps * v)) / (2 * eps)
            fd_g = (F_gpu(prim + eps * v) - F_gpu(prim - eps * v)) / (2 * eps)
            assert abs(adj - fd_o) <= tol * abs(fd_o), (trial, adj, fd_o)
            assert abs(adj - fd_g) <= tol * abs(fd_g), (trial, adj, fd_g)


def _noisy_blast(m, noise=1e-6):
    """The blast workload with relative noise 1e-6 on every primitive (absolute
    1e-6 on the components that vanish).  The exact blast sits on the
    switches of the scheme: its symmetric states put cluster memberships,
    the frame alignment (|B_t| at the 1e-10 threshold) and Y (exactly zero
    jumps) where a perturbation decides them, and its recorded map jumps by
    ~1e-11 under perturbations of any size; the noise moves every state off
    those switches, far below any physical scale."""
    x, prim = wl.blast3_config(m)
    r = wl.rng(700)
    prim = prim * (1.0 + noise * r.standard_normal(prim.shape))
    for c in (1, 2, 3, 6, 7):
        prim[c] += noise * r.standard_normal(prim.shape[1:])
    return x, np.ascontiguousarray(prim)


def _blast_check(m, cases, steps=20, eps=1e-6):
    x, prim = _noisy_blast(m)
    r0 = np.sqrt((x ** 2).sum(axis=0))
    with esmm.Grid3((m, m, m), (-0.5,) * 3, (0.5,) * 3, bc=(1, 1, 1), p=2, w=5) as g:
        g.state_set(prim, x)
        g.adjoint_record(steps)
        xf = g.state_get(esmm.GET_X)
        for comp, dname, tol in cases:
            wts, inside = _box_weights(xf, 0.0, 0.2)
            assert inside.sum() > 0
            if comp != 0:
                wts[comp], wts[0] = wts[0], 0.0
            _, lam_prim = g.adjoint_vjp(wts)
            assert np.isfinite(lam_prim).all()

            def F(pr):
                g.state_set(pr, x)
                g.adjoint_replay(steps)
                return float((wts * g.state_get(esmm.GET_CONS)).sum())

            v = np.zeros_like(prim)
            v[4] = prim[4] * (r0 < 0.1) if dname == "inside" else prim[4]
            adj = float((lam_prim * v).sum())
            fd = (F(prim + eps * v) - F(prim - eps * v)) / (2 * eps)
            if abs(adj - fd) > tol * abs(fd):
                # the central difference's own uncertainty, from halving its
                # step: where the perturbed runs cross one of the recorded
                # map's switch points (the sign switch, a cluster or frame
                # threshold) the difference quotient moves with eps, and the
                # comparison can be no sharper
                fd2 = (F(prim + 0.5 * eps * v) - F(prim - 0.5 * eps * v)) / eps
                unc = 2.0 * abs(fd - fd2)
                assert abs(adj - fd) <= tol * abs(fd) + unc, (comp, dname, adj, fd, fd2)
            else:
                assert abs(adj - fd) <= tol * abs(fd), (comp, dname, adj, fd)


def test_blast_adjoint_against_fd():
    # the functional of the 128^3 workload (J D over [0, 0.2]^3) and J E over
    # the same box, along the pressure inside the sphere and everywhere
    _blast_check(32, [(0, "inside", 1e-3), (0, "all", 1e-3), (4, "inside", 1e-6), (4, "all", 1e-6)])


def test_blast_adjoint_full_size():
    # 128^3, 20 recorded steps with checkpoints, gradient with respect to the
    # initial pressure.  J D over [0, 0.2]^3 hardly changes in these steps
    # (no wave reaches the box's outer faces, and no mass crosses the
    # symmetry planes), so the check uses J E over the box, which the blast
    # changes at first order
    _blast_check(128, [(4, "inside", 1e-5)])
