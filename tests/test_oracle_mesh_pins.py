"""Pins of the oracle's Sec. 5 mesh iteration by what the mathematics fixes.

  * the low-pass filter of the Sec. 5 remark is a convolution with a
    separable kernel (1/4, 1/2, 1/4) per direction, so a Fourier mode
    cos(theta . i) is an eigenfunction with multiplier prod_d (1 + cos
    theta_d)/2 per pass; with zero-gradient ends the half-sample cosine
    modes cos(theta (i + 1/2)), theta = pi m / n, are eigenfunctions with the
    same multiplier;
  * with a uniform monitor one Jacobi sweep of the mesh equations replaces a
    node by the mean of its 2d neighbours, so a mode sin(theta . i) added to
    a uniform mesh is multiplied by sum_d cos(theta_d) / d;
  * the iteration's fixed point solves the Euler-Lagrange equations of the
    adaption functional (eq. mesh_func with G_k = omega I): with omega
    depending on i only, that is 1-D equidistribution, (omega_i +
    omega_{i+1})(x_{i+1} - x_i) = const; in general it is the minimiser of
    the discrete energy sum over mesh edges of (omega_a + omega_b)/2 |x_b -
    x_a|^2 with the boundary nodes held, assembled here edge by edge and
    solved as a sparse linear system.
"""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import workloads as wl


def _cfg2(nx, ny, bc, period=(1.0, 1.0)):
    return oracle.make_cfg(nx, ny, bc=bc, period=period)


def _cfg3(nx, ny, nz, bc, period=(1.0, 1.0, 1.0)):
    return oracle.make_cfg3(nx, ny, nz, bc=bc, period=period)


# ------------------------------------------------------------------ the filter
@pytest.mark.parametrize("passes", [1, 4])
def test_filter_multiplies_a_periodic_mode_by_its_symbol(passes):
    nx, ny = 24, 20
    tx, ty = 2 * np.pi * 3 / nx, 2 * np.pi * 5 / ny
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    eps = 0.3
    om = 1.0 + eps * np.cos(tx * i + 0.4) * np.cos(ty * j - 1.1)
    cfg = _cfg2(nx, ny, (oracle.PERIODIC, oracle.PERIODIC))
    out = oracle.mesh_filter(cfg, om, passes)
    g = ((1 + np.cos(tx)) / 2 * (1 + np.cos(ty)) / 2) ** passes
    want = 1.0 + g * eps * np.cos(tx * i + 0.4) * np.cos(ty * j - 1.1)
    assert np.abs(out - want).max() < 1e-14


def test_filter_keeps_half_sample_cosines_at_outflow_ends():
    # ghosts copy the end node, omega_{-1} = omega_0: the half-sample cosine
    # modes satisfy that reflection at both ends
    nx, ny = 17, 13
    tx, ty = np.pi * 4 / nx, np.pi * 3 / ny
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    mode = np.cos(tx * (i + 0.5)) * np.cos(ty * (j + 0.5))
    cfg = _cfg2(nx, ny, (oracle.OUTFLOW, oracle.OUTFLOW))
    out = oracle.mesh_filter(cfg, 2.0 + 0.5 * mode, 3)
    g = ((1 + np.cos(tx)) / 2 * (1 + np.cos(ty)) / 2) ** 3
    assert np.abs(out - (2.0 + 0.5 * g * mode)).max() < 1e-14


def test_filter_symbol_in_3d():
    nx, ny, nz = 12, 10, 8
    th = [2 * np.pi * 2 / nx, 2 * np.pi * 3 / ny, np.pi * 3 / nz]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = np.cos(th[0] * i) * np.sin(th[1] * j + 0.3) * np.cos(th[2] * (k + 0.5))
    cfg = _cfg3(nx, ny, nz, (oracle.PERIODIC, oracle.PERIODIC, oracle.OUTFLOW))
    out = oracle.mesh_filter3(cfg, 1.5 + 0.4 * mode, 2)
    g = np.prod([(1 + np.cos(t)) / 2 for t in th]) ** 2
    assert np.abs(out - (1.5 + 0.4 * g * mode)).max() < 1e-14


# ------------------------------------------------------------- Jacobi, one sweep
@pytest.mark.parametrize("sweeps", [1, 3])
def test_jacobi_damps_a_mode_by_the_neighbour_mean(sweeps):
    nx, ny = 20, 16
    Lx, Ly = 2.0, 1.5
    tx, ty = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    base = np.stack([i * Lx / nx - 1.0, j * Ly / ny + 0.25])
    d = 1e-2
    pert = np.stack([d * np.sin(tx * i + ty * j), -0.5 * d * np.cos(tx * i) * np.sin(ty * j)])
    cfg = _cfg2(nx, ny, (oracle.PERIODIC, oracle.PERIODIC), period=(Lx, Ly))
    om = np.full((ny, nx), 2.7)
    X = oracle.mesh_jacobi(cfg, om, base + pert, sweeps)
    # sin(a i + b j) and cos(a i) sin(b j) are both eigenfunctions of the mean
    # of the four neighbours with eigenvalue (cos a + cos b) / 2
    g = ((np.cos(tx) + np.cos(ty)) / 2) ** sweeps
    assert np.abs(X - (base + g * pert)).max() < 1e-15


def test_jacobi_damps_a_mode_by_the_neighbour_mean_in_3d():
    nx, ny, nz = 10, 8, 6
    th = [2 * np.pi / nx, 2 * np.pi * 2 / ny, 2 * np.pi / nz]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([i / nx, j / ny, k / nz])
    pert = 1e-2 * np.stack([np.sin(th[0] * i) * np.cos(th[2] * k), np.sin(th[1] * j), np.cos(th[2] * k)])
    cfg = _cfg3(nx, ny, nz, (oracle.PERIODIC,) * 3)
    om = np.full((nz, ny, nx), 0.8)
    X = oracle.mesh_jacobi3(cfg, om, base + pert, 1)
    c = [np.cos(t) for t in th]
    # component 0 varies along i and k, component 1 along j, component 2 along k
    gains = [(c[0] + 1 + c[2]) / 3, (1 + c[1] + 1) / 3, (1 + 1 + c[2]) / 3]
    want = base + np.stack([gains[a] * pert[a] for a in range(3)])
    assert np.abs(X - want).max() < 1e-15


# ------------------------------------------------------ the fixed point (EL eqs)
def _equidistributed(om_i, a, b):
    """1-D equidistribution on fixed ends a, b: spacing proportional to
    1/(omega_i + omega_{i+1})."""
    h = 1.0 / (om_i[:-1] + om_i[1:])
    return a + (b - a) * np.concatenate([[0.0], np.cumsum(h)]) / h.sum()


def test_jacobi_converges_to_1d_equidistribution():
    nx, ny = 14, 6
    r = wl.rng(5)
    om_i = np.sqrt(1.0 + 20.0 * r.uniform(0, 1, nx))
    om = np.broadcast_to(om_i, (ny, nx)).copy()
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    x0 = np.stack([i / (nx - 1.0), j / ny])
    cfg = _cfg2(nx, ny, (oracle.OUTFLOW, oracle.PERIODIC), period=(1.0, 1.0))
    X = oracle.mesh_jacobi(cfg, om, x0, 3000)
    want = _equidistributed(om_i, 0.0, 1.0)
    assert np.abs(X[0] - want[None, :]).max() < 1e-13
    assert np.abs(X[1] - x0[1]).max() < 1e-15
    # the Euler-Lagrange flux (omega_i + omega_{i+1}) dx is the same on every edge
    flux = (om_i[:-1] + om_i[1:]) * np.diff(X[0][0])
    assert np.ptp(flux) < 1e-12 * flux.mean()


def test_jacobi_converges_to_1d_equidistribution_in_3d():
    nx, ny, nz = 12, 4, 4
    om_i = 1.0 + 3.0 * np.sin(np.pi * np.arange(nx) / (nx - 1)) ** 2
    om = np.broadcast_to(om_i, (nz, ny, nx)).copy()
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x0 = np.stack([2.0 * i / (nx - 1.0) - 1.0, j / ny, k / nz])
    cfg = _cfg3(nx, ny, nz, (oracle.OUTFLOW, oracle.PERIODIC, oracle.PERIODIC))
    X = oracle.mesh_jacobi3(cfg, om, x0, 4000)
    want = _equidistributed(om_i, -1.0, 1.0)
    assert np.abs(X[0] - want[None, None, :]).max() < 1e-13
    assert np.abs(X[1:] - x0[1:]).max() < 1e-15


def _energy_minimiser(om, x0, fixed):
    """Minimise sum over edges (a, b) of the 2D index grid of
    (om_a + om_b)/2 (x_b - x_a)^2 over the free nodes, with the fixed nodes
    held at x0 (one coordinate): the normal equations assembled edge by
    edge."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    ny, nx = om.shape
    N = nx * ny
    rows, cols, vals = [], [], []
    edges = [((j, i), (j, i + 1)) for j in range(ny) for i in range(nx - 1)]
    edges += [((j, i), (j + 1, i)) for j in range(ny - 1) for i in range(nx)]
    for (ja, ia), (jb, ib) in edges:
        a, b = ja * nx + ia, jb * nx + ib
        wgt = 0.5 * (om[ja, ia] + om[jb, ib])
        # gradient of wgt (x_b - x_a)^2 / 2 ... times 2: the Hessian block
        rows += [a, a, b, b]
        cols += [a, b, a, b]
        vals += [wgt, -wgt, -wgt, wgt]
    H = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    free = ~fixed.ravel()
    xf = x0.ravel().copy()
    rhs = -H[free][:, ~free] @ xf[~free]
    xf[free] = spl.spsolve(H[free][:, free].tocsc(), rhs)
    return xf.reshape(ny, nx)


def test_jacobi_fixed_point_minimises_the_discrete_adaption_energy():
    nx, ny = 12, 10
    r = wl.rng(8)
    om = np.sqrt(1.0 + 30.0 * r.uniform(0, 1, (ny, nx)))
    x0 = wl.random_mesh(nx, ny, r, amp=0.2, periodic=(False, False))
    cfg = _cfg2(nx, ny, (oracle.OUTFLOW, oracle.OUTFLOW))
    X = oracle.mesh_jacobi(cfg, om, x0, 4000)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    fixed = (i == 0) | (i == nx - 1) | (j == 0) | (j == ny - 1)
    for c in range(2):
        want = _energy_minimiser(om, x0[c], fixed)
        assert np.abs(X[c] - want).max() < 1e-13, c
