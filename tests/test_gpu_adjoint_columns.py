"""The adjoint's vector-Jacobian product element by element against the
oracle's Jacobian, column by column.

lambda = (d rhs/d cons)^T mu from the adjoint kernels is compared entry by
entry with sum_i mu_i (rhs_i(cons + h e_j) - rhs_i(cons - h e_j)) / 2h, the
oracle's right-hand side differenced along each unit vector e_j (h = 1e-6 of
the entry, at least 1e-8 of its component's largest magnitude; halving h
moves these columns by < 1e-7 of their largest entry on these states):

  * 2D RHD, EC (p = 2) and ES (p = 2, WENO5): every column, mu random on the
    whole grid;
  * 2D RMHD and 3D RMHD, ES (p = 2, WENO5): mu random at two nodes only.
    The columns inside the union of the two nodes' stencils (crosses of
    radius 3 along the grid lines) are differenced; outside it lambda must
    be exactly 0, as the right-hand side at a node reads no other nodes.

Smooth periodic states on curvilinear meshes with a mesh velocity, where no
decision of the sign switch Y flips within +-h.
"""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import esmm
from paper_2107_12027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
G43 = 4.0 / 3.0
REL_STEP = 1.0e-6
TOL = 1.0e-6


def _fd_entry(f, cons, mu, idx, scale):
    h = REL_STEP * max(abs(cons[idx]), 1e-2 * scale[idx[0]])
    up = cons.copy()
    up[idx] += h
    dn = cons.copy()
    dn[idx] -= h
    return float((mu * (f(up) - f(dn))).sum()) / (2.0 * h)


def _stencil_nodes(dims, centres, radius):
    out = set()
    for nd in centres:
        out.add(nd)
        for ax in range(len(dims)):
            for k in range(1, radius + 1):
                for s in (-1, 1):
                    q = list(nd)
                    q[ax] = (q[ax] + s * k) % dims[ax]
                    out.add(tuple(q))
    return sorted(out)


def _compare(lam, f, cons, mu, nodes):
    scale = np.abs(cons).reshape(cons.shape[0], -1).max(axis=1)
    ref = np.zeros_like(cons)
    for nd in nodes:
        for c in range(cons.shape[0]):
            ref[(c,) + nd] = _fd_entry(f, cons, mu, (c,) + nd, scale)
    inside = np.zeros(cons.shape, dtype=bool)
    for nd in nodes:
        inside[(slice(None),) + nd] = True
    err = np.abs(lam - ref)[inside].max() / np.abs(ref).max()
    assert err <= TOL, err
    return inside


@pytest.mark.parametrize("w", [0, 5])
def test_rhd_vjp_every_column(w):
    n, m = 12, 10
    x = wl.wavy_mesh(n, m, amp=0.03)
    xd = np.ascontiguousarray(wl.wavy_mesh_velocity(n, m, amp=0.03, t=1.0))
    prim = wl.smooth_random_state(x, wl.rng(300))
    cfg = oracle.make_cfg(n, m, p=2, w=w)
    cons, J = oracle.init_state(cfg, prim, x)
    mu = wl.rng(310 + w).standard_normal(cons.shape)
    with esmm.Grid((n, m), p=2, w=w) as g:
        lam = g.rhs_vjp(cons, J, x, xd, mu)
    nodes = [(j, i) for j in range(m) for i in range(n)]
    _compare(lam, lambda c: oracle.rhs(cfg, c, J, x, xd)[0], cons, mu, nodes)


def _two_node_mu(cons, seed):
    r = wl.rng(seed)
    dims = cons.shape[1:]
    centres = []
    while len(centres) < 2:
        nd = tuple(int(r.integers(0, d)) for d in dims)
        if nd not in centres:
            centres.append(nd)
    mu = np.zeros_like(cons)
    for nd in centres:
        mu[(slice(None),) + nd] = r.standard_normal(cons.shape[0])
    return mu, centres


def test_rmhd_vjp_columns_of_two_stencils():
    n, m = 12, 10
    x = wl.wavy_mesh(n, m, amp=0.03)
    xd = np.ascontiguousarray(wl.wavy_mesh_velocity(n, m, amp=0.03, t=1.0))
    prim = wl.smooth_random_state_mhd(x, wl.rng(600))
    cfg = oracle.make_cfg(n, m, p=2, w=5, gamma=G43, phys=oracle.RMHD)
    cons, J = oracle.init_state(cfg, prim, x)
    mu, centres = _two_node_mu(cons, 620)
    with esmm.Grid((n, m), p=2, w=5, gamma=G43, phys=esmm.RMHD) as g:
        lam = g.rhs_vjp(cons, J, x, xd, mu)
    nodes = _stencil_nodes(cons.shape[1:], centres, 3)
    inside = _compare(lam, lambda c: oracle.rhs(cfg, c, J, x, xd)[0], cons, mu, nodes)
    assert np.all(lam[~inside] == 0.0)


def test_rmhd3d_vjp_columns_of_two_stencils():
    n = (8, 7, 6)
    x = wl.wavy_mesh3(n, amp=0.04)
    xd = np.ascontiguousarray(wl.wavy_mesh_velocity3(n, amp=0.04, t=1.2))
    prim = wl.smooth_random_state_mhd3(x, wl.rng(650))
    cfg = oracle.make_cfg3(*n, p=2, w=5)
    cons, J = oracle.init_state3(cfg, prim, x)
    mu, centres = _two_node_mu(cons, 660)
    with esmm.Grid3(n, p=2, w=5) as g:
        lam = g.rhs_vjp(cons, J, x, xd, mu)
    nodes = _stencil_nodes(cons.shape[1:], centres, 3)
    inside = _compare(lam, lambda c: oracle.rhs3(cfg, c, J, x, xd)[0], cons, mu, nodes)
    assert np.all(lam[~inside] == 0.0)
