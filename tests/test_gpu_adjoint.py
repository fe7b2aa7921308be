"""Adjoint (vector-Jacobian products) against finite differences.

  * (d rhs/d cons)^T mu from the adjoint kernels against central differences
    of the GPU right-hand side and of the oracle's, in random directions;
  * the gradient of a final-time functional (integrated J (D + E) over a
    sub-box) with respect to the initial pressure, through several recorded SSP-RK3
    steps with per-step checkpoints, against central differences of the
    oracle's steps with the recorded mesh velocities and time steps.  The EC
    scheme's map is smooth and is held to 1e-6.  The ES scheme's is not
    differentiable where the sign switch Y flips: where a jump [[V~]] crosses
    zero while the WENO jump does not, the flux jumps by that WENO jump.  The
    adjoint differentiates with Y frozen, so central differences that
    straddle such a flip differ from it; the ES case is held to 5e-2.
  * the torch.autograd wrapper gives the same gradient.
"""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _smooth_case(n=24, m=20, seed=300):
    x = wl.wavy_mesh(n, m, amp=0.03)
    xdot = wl.wavy_mesh_velocity(n, m, amp=0.03, t=1.0)
    prim = wl.smooth_random_state(x, wl.rng(seed))
    return x, np.ascontiguousarray(xdot), prim


@pytest.mark.parametrize("p,w", [(2, 0), (2, 5), (3, 5), (1, 3)])
def test_rhs_vjp_against_finite_differences(p, w):
    n, m = 24, 20
    x, xdot, prim = _smooth_case(n, m)
    cfg = oracle.make_cfg(n, m, p=p, w=w)
    cons, J = oracle.init_state(cfg, prim, x)
    r = wl.rng(301)
    mu = r.standard_normal((4, m, n))
    with esmm.Grid((n, m), p=p, w=w) as g:
        lam = g.rhs_vjp(cons, J, x, xdot, mu)
        for trial in range(3):
            v = r.standard_normal((4, m, n)) * np.abs(cons) * 1e-2
            eps = 1e-5
            adj = float((lam * v).sum())
            dg = (g.rhs(cons + eps * v, J, x, xdot)[0] - g.rhs(cons - eps * v, J, x, xdot)[0]) / (2 * eps)
            do = (oracle.rhs(cfg, cons + eps * v, J, x, xdot)[0] - oracle.rhs(cfg, cons - eps * v, J, x, xdot)[0]) / (2 * eps)
            fd_gpu, fd_ora = float((mu * dg).sum()), float((mu * do).sum())
            assert abs(adj - fd_gpu) <= 1e-6 * abs(fd_gpu), (trial, adj, fd_gpu)
            assert abs(adj - fd_ora) <= 1e-6 * abs(fd_ora), (trial, adj, fd_ora)


def _functional_weights(x, box, energy=False):
    """Weights of a functional sum w . cons: J D over the box (and J E with
    energy=True, whose pressure derivative is O(1), so that central
    differences resolve it after steps short enough to leave the mass almost
    unchanged)."""
    w = np.zeros((4,) + x.shape[1:])
    inside = (x[0] >= box[0]) & (x[0] <= box[1]) & (x[1] >= box[2]) & (x[1] <= box[3])
    w[0][inside] = 1.0
    if energy:
        w[3][inside] = 1.0
    return w


@pytest.mark.parametrize("case,w,tol", [("smooth", 0, 1e-6), ("riemann", 0, 1e-6), ("smooth", 5, 5e-2)])
def test_multistep_adjoint_against_oracle_fd(case, w, tol):
    steps = 4
    if case == "smooth":
        n = 28
        x, prim = wl.sine_config(n)
        prim = wl.smooth_random_state(x, wl.rng(310))
        kw = dict(bc=(0, 0), lo=(0, 0), hi=(1, 1))
        ocfg = dict(bc=(0, 0), period=(1.0, 1.0))
        box = (0.0, 0.3, 0.0, 0.3)
    else:
        n = 32
        x, prim = wl.batch_problem(3, n)
        kw = dict(bc=(1, 1), lo=(-1, -1), hi=(1, 1))
        ocfg = dict(bc=(1, 1), period=(2.0, 2.0))
        box = (-0.2, 0.4, -0.3, 0.3)
    params = dict(alpha=200.0, monitor=esmm.MONITOR_LNRHO)
    with esmm.Grid((n, n), kw["lo"], kw["hi"], bc=kw["bc"], p=2, w=w, **params) as g:
        g.state_set(prim, x)
        g.adjoint_record(steps)
        dts = g.adjoint_steps()
        xdots = [g.adjoint_checkpoint(k, esmm.GET_XDOT) for k in range(steps)]
        wts = _functional_weights(g.state_get(esmm.GET_X), box, energy=True)
        _, lam_prim = g.adjoint_vjp(wts)
        # the functional through the recorded map, on the oracle
        cfg = oracle.make_cfg(n, n, p=2, w=w, alpha=200.0, **ocfg)

        def F_oracle(pr):
            cons, J = oracle.init_state(cfg, pr, x)
            xs = x
            for k in range(steps):
                cons, J, xs = oracle.rk_step_given(cfg, cons, J, xs, xdots[k], dts[k])
            return float((wts * cons).sum())

        def F_gpu(pr):
            g.state_set(pr, x)
            g.adjoint_replay(steps)
            return float((wts * g.state_get(esmm.GET_CONS)).sum())

        r = wl.rng(311)
        for trial in range(2):
            v = np.zeros_like(prim)
            v[3] = r.standard_normal(prim.shape[1:]) * prim[3]      # pressure direction
            eps = 1e-6
            adj = float((lam_prim * v).sum())
            fd_o = (F_oracle(prim + eps * v) - F_oracle(prim - eps * v)) / (2 * eps)
            fd_g = (F_gpu(prim + eps * v) - F_gpu(prim - eps * v)) / (2 * eps)
            assert abs(adj - fd_o) <= tol * abs(fd_o), (trial, adj, fd_o)
            assert abs(adj - fd_g) <= tol * abs(fd_g), (trial, adj, fd_g)


def test_autograd_function_gradient():
    torch = pytest.importorskip("torch")
    from paper_2107_12027_gb300.autograd import RKSteps
    n = 24
    x, prim = wl.sine_config(n)
    prim = wl.smooth_random_state(x, wl.rng(320))
    dev = torch.device("cuda", 0)
    with esmm.Grid((n, n), p=2, w=5, alpha=20.0, monitor=esmm.MONITOR_RHO) as g:
        p0 = torch.tensor(prim, device=dev, requires_grad=True)
        xt = torch.tensor(x, device=dev)
        wts = torch.tensor(_functional_weights(x, (0.0, 0.5, 0.0, 0.5)), device=dev)
        out = RKSteps.apply(p0, g, xt, 3, 0.0)
        F = (wts * out).sum()
        F.backward()
        grad = p0.grad.cpu().numpy()
        _, lam_prim = g.adjoint_vjp(wts.cpu().numpy())
        np.testing.assert_allclose(grad, lam_prim, rtol=1e-12, atol=1e-14 * np.abs(lam_prim).max())
        assert np.abs(grad[3]).max() > 0.0
