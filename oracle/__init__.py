"""FP64 CPU oracle for the ES adaptive moving-mesh scheme (2D RHD and RMHD).

TEST INFRASTRUCTURE.  This package is the independent checker of the CUDA
library: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it.  It shares no code with the CUDA path; the C
sources ``esmm_oracle.c`` (2D grid, mesh, RHD), ``esmm_oracle_mhd.c``
(pointwise RMHD) and ``esmm_oracle3d.c`` (3D RMHD grid) restate the paper (Duan & Tang, arXiv 2107.12027)
one node, pair and interface at a time.

Array conventions match the C header: structure of arrays, ``[comp][j][i]``
with ``i`` fastest, FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "esmm_oracle.c"), os.path.join(_HERE, "esmm_oracle_mhd.c"),
         os.path.join(_HERE, "esmm_oracle3d.c")]
_HDR = os.path.join(_HERE, "esmm_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, OUTFLOW, INFLOW = 0, 1, 2
MONITOR_RHO, MONITOR_LNRHO = 0, 1
RHD, RMHD = 0, 1


class Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("bc", ctypes.c_int * 2),
        ("period", ctypes.c_double * 2),
        ("gamma", ctypes.c_double),
        ("p", ctypes.c_int), ("w", ctypes.c_int),
        ("weno_eps", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("monitor", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("n_filter", ctypes.c_int),
        ("mu", ctypes.c_int),
        ("move_mesh", ctypes.c_int),
        ("phys", ctypes.c_int),
        ("alpha_lap", ctypes.c_double),
        ("inflow", ctypes.c_double * 8),
    ]


class Cfg3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("period", ctypes.c_double * 3),
        ("gamma", ctypes.c_double),
        ("p", ctypes.c_int), ("w", ctypes.c_int),
        ("weno_eps", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("monitor", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("n_filter", ctypes.c_int),
        ("mu", ctypes.c_int),
        ("move_mesh", ctypes.c_int),
        ("alpha_lap", ctypes.c_double),
        ("inflow", ctypes.c_double * 8),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newer = (os.path.exists(_LIB)
             and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in _SRCS + [_HDR]))
    if force or not newer:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        # -ffp-contract=off: every product and sum is rounded as written.
        # -fopenmp: the per-node and per-interface loops run on all host
        # threads; every reduction across threads is a max or a min, so the
        # results equal the single-threaded ones bit for bit.
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            # idle OpenMP threads sleep instead of spinning: the tests make
            # thousands of small calls, between which spinning threads would
            # only compete with the caller
            os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
            L = ctypes.CDLL(path)
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.POINTER(ctypes.c_int)
            c = ctypes.POINTER(Cfg)
            c3 = ctypes.POINTER(Cfg3)
            sig = {
                "oref_set_threads": (ctypes.c_int, [ctypes.c_int]),
                "oref_alpha": (None, [ctypes.c_int, d]),
                "oref_logmean": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
                "oref_prim2cons": (None, [ctypes.c_double, d, d]),
                "oref_cons2prim": (ctypes.c_int, [ctypes.c_double, d, d, i]),
                "oref_flux": (None, [ctypes.c_double, d, ctypes.c_int, d]),
                "oref_entropy": (ctypes.c_double, [ctypes.c_double, d]),
                "oref_entropy_vars": (None, [ctypes.c_double, d, d]),
                "oref_potentials": (None, [d, d, d]),
                "oref_ec_flux": (None, [ctypes.c_double, d, d, d, d, d]),
                "oref_eigen": (None, [ctypes.c_double, d, d, d]),
                "oref_weno": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, d]),
                "oref_metrics": (None, [c, d, d, d]),
                "oref_rhs": (ctypes.c_int, [c, d, d, d, d, d, d]),
                "oref_cfl_dt": (ctypes.c_int, [c, d, d, d, d]),
                "oref_monitor": (ctypes.c_int, [c, d, d, d]),
                "oref_cfl_solve": (ctypes.c_double, [ctypes.c_int, ctypes.c_long, ctypes.c_double, d, d, d,
                                                     ctypes.c_double, d, i]),
                "oref_filter": (None, [c, d, ctypes.c_int]),
                "oref_jacobi": (None, [c, d, d, ctypes.c_int, d]),
                "oref_mesh": (ctypes.c_int, [c, d, d, d, ctypes.c_double, d, d, d]),
                "oref_rk_step": (ctypes.c_int, [c, d, d, d, ctypes.c_double, d]),
                "oref_rk_step_given": (ctypes.c_int, [c, d, d, d, d, ctypes.c_double]),
                "oref_init_state": (ctypes.c_int, [c, d, d, d, d]),
                "oref_state_prim": (ctypes.c_int, [c, d, d, d]),
                "oref_totals": (ctypes.c_int, [c, d, d, d, d, d]),
                "oref_mhd_prim2cons": (None, [ctypes.c_double, d, d]),
                "oref_mhd_flux": (None, [ctypes.c_double, d, ctypes.c_int, d]),
                "oref_mhd_cons2prim": (ctypes.c_int, [ctypes.c_double, d, d, i]),
                "oref_mhd_entropy": (ctypes.c_double, [ctypes.c_double, d]),
                "oref_mhd_entropy_vars": (None, [ctypes.c_double, d, d]),
                "oref_mhd_potentials": (None, [d, d, d, d]),
                "oref_mhd_phiprime": (None, [d, d]),
                "oref_mhd_ec_flux": (None, [ctypes.c_double, d, d, d, d]),
                "oref_mhd_eigen": (None, [ctypes.c_double, d, d, d]),
                "oref3_metrics": (None, [c3, d, d, d]),
                "oref3_init_state": (ctypes.c_int, [c3, d, d, d, d]),
                "oref3_state_prim": (ctypes.c_int, [c3, d, d, d]),
                "oref3_rhs": (ctypes.c_int, [c3, d, d, d, d, d, d]),
                "oref3_cfl_dt": (ctypes.c_int, [c3, d, d, d, d]),
                "oref3_monitor": (ctypes.c_int, [c3, d, d, d]),
                "oref3_filter": (None, [c3, d, ctypes.c_int]),
                "oref3_jacobi": (None, [c3, d, d, ctypes.c_int, d]),
                "oref3_mesh": (ctypes.c_int, [c3, d, d, d, ctypes.c_double, d, d, d]),
                "oref3_rk_step": (ctypes.c_int, [c3, d, d, d, ctypes.c_double, d]),
                "oref3_rk_step_given": (ctypes.c_int, [c3, d, d, d, d, ctypes.c_double]),
                "oref3_totals": (ctypes.c_int, [c3, d, d, d, d, d]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (n <= 0: all host threads);
    returns the number in effect.  Results do not depend on it."""
    return lib().oref_set_threads(int(n))


def make_cfg(nx, ny, bc=(PERIODIC, PERIODIC), period=(1.0, 1.0), gamma=5.0 / 3.0,
             p=2, w=5, weno_eps=1e-6, cfl=0.4, monitor=MONITOR_LNRHO, alpha=20.0,
             n_filter=4, mu=10, move_mesh=1, phys=RHD, alpha_lap=0.0, inflow=None) -> Cfg:
    c = Cfg()
    c.nx, c.ny = nx, ny
    c.bc[0], c.bc[1] = bc
    c.period[0], c.period[1] = period
    c.gamma, c.p, c.w, c.weno_eps, c.cfl = gamma, p, w, weno_eps, cfl
    c.monitor, c.alpha, c.n_filter, c.mu, c.move_mesh = monitor, alpha, n_filter, mu, move_mesh
    c.phys, c.alpha_lap = phys, alpha_lap
    for a, v in enumerate(inflow if inflow is not None else ()):
        c.inflow[a] = v
    return c


def nvar(cfg):
    """Number of unknowns per node: 4 (RHD) or 8 (RMHD)."""
    return 8 if cfg.phys == RMHD else 4


# ---- pointwise functions ---------------------------------------------------
def alpha(p):
    out = np.zeros(p)
    lib().oref_alpha(p, _p(out))
    return out


def logmean(a, b):
    return lib().oref_logmean(float(a), float(b))


def prim2cons(gamma, w):
    w = _vec(w, 4)
    U = np.zeros(4)
    lib().oref_prim2cons(gamma, _p(w), _p(U))
    return U


def cons2prim(gamma, U):
    U = _vec(U, 4)
    w = np.zeros(4)
    it = ctypes.c_int(0)
    st = lib().oref_cons2prim(gamma, _p(U), _p(w), ctypes.byref(it))
    return w, st, it.value


def flux(gamma, w, direction):
    w = _vec(w, 4)
    F = np.zeros(4)
    lib().oref_flux(gamma, _p(w), direction, _p(F))
    return F


def entropy(gamma, w):
    return lib().oref_entropy(gamma, _p(_vec(w, 4)))


def entropy_vars(gamma, w):
    V = np.zeros(4)
    lib().oref_entropy_vars(gamma, _p(_vec(w, 4)), _p(V))
    return V


def potentials(w):
    phi = np.zeros(1)
    psi = np.zeros(2)
    lib().oref_potentials(_p(_vec(w, 4)), _p(phi), _p(psi))
    return phi[0], psi


def ec_flux(gamma, wl, wr):
    Ut, F1, F2 = np.zeros(4), np.zeros(4), np.zeros(4)
    lib().oref_ec_flux(gamma, _p(_vec(wl, 4)), _p(_vec(wr, 4)), _p(Ut), _p(F1), _p(F2))
    return Ut, F1, F2


def eigen(gamma, w_rot):
    lam, R = np.zeros(4), np.zeros(16)
    lib().oref_eigen(gamma, _p(_vec(w_rot, 4)), _p(lam), _p(R))
    return lam, R.reshape(4, 4)


def weno(w, eps, s):
    s = _vec(s, w)
    return lib().oref_weno(w, eps, _p(s))


# ---- grid functions --------------------------------------------------------
def metrics(cfg, x):
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    x = _vec(x, 2 * N)
    m = np.zeros(4 * N)
    J0 = np.zeros(N)
    lib().oref_metrics(ctypes.byref(cfg), _p(x), _p(m), _p(J0))
    return m.reshape(4, cfg.ny, cfg.nx), J0.reshape(cfg.ny, cfg.nx)


def init_state(cfg, prim, x):
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    prim, x = _vec(prim, nv * N), _vec(x, 2 * N)
    cons, J = np.zeros(nv * N), np.zeros(N)
    lib().oref_init_state(ctypes.byref(cfg), _p(prim), _p(x), _p(cons), _p(J))
    return cons.reshape(nv, cfg.ny, cfg.nx), J.reshape(cfg.ny, cfg.nx)


def state_prim(cfg, cons, J):
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    prim = np.zeros(nv * N)
    st = lib().oref_state_prim(ctypes.byref(cfg), _p(_vec(cons, nv * N)), _p(_vec(J, N)), _p(prim))
    return prim.reshape(nv, cfg.ny, cfg.nx), st


def rhs(cfg, cons, J, x, xdot=None):
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    if xdot is None:
        xdot = np.zeros(2 * N)
    dcons, dJ = np.zeros(nv * N), np.zeros(N)
    st = lib().oref_rhs(ctypes.byref(cfg), _p(_vec(cons, nv * N)), _p(_vec(J, N)),
                        _p(_vec(x, 2 * N)), _p(_vec(xdot, 2 * N)), _p(dcons), _p(dJ))
    if st != 0:
        raise RuntimeError("oracle rhs: cons2prim failed")
    return dcons.reshape(nv, cfg.ny, cfg.nx), dJ.reshape(cfg.ny, cfg.nx)


def cfl_dt(cfg, cons, J, x):
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    dt = np.zeros(1)
    st = lib().oref_cfl_dt(ctypes.byref(cfg), _p(_vec(cons, nv * N)), _p(_vec(J, N)),
                           _p(_vec(x, 2 * N)), _p(dt))
    if st != 0:
        raise RuntimeError("oracle cfl: cons2prim failed")
    return dt[0]


def monitor(cfg, cons, J):
    """Sec. 5 monitor omega [ny][nx] before the low-pass filter (with the
    Laplacian term of the vortex example when cfg.alpha_lap > 0)."""
    N = cfg.nx * cfg.ny
    om = np.zeros(N)
    st = lib().oref_monitor(ctypes.byref(cfg), _p(_vec(cons, nvar(cfg) * N)), _p(_vec(J, N)), _p(om))
    if st != 0:
        raise RuntimeError("oracle monitor: cons2prim failed")
    return om.reshape(cfg.ny, cfg.nx)


def cfl_solve(a, bmin, bmax, cfl, tau, dt_given=0.0):
    """The step of eq. cfl with the mesh velocity in the spectral radius from
    the per-node terms a, bmin, bmax [ndir][N]: returns (dt, tau used, Newton
    steps, -1 for the fallback)."""
    a, bmin, bmax = (np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in (a, bmin, bmax))
    ndir, N = a.shape
    t = ctypes.c_double(tau)
    it = ctypes.c_int(0)
    dt = lib().oref_cfl_solve(ndir, N, float(cfl), _p(a), _p(bmin), _p(bmax), float(dt_given), ctypes.byref(t),
                              ctypes.byref(it))
    return dt, t.value, it.value


def mesh_filter(cfg, om, n):
    """The Sec. 5 low-pass filter applied n times to om [ny][nx] (a copy)."""
    N = cfg.nx * cfg.ny
    om = _vec(om, N).copy()
    lib().oref_filter(ctypes.byref(cfg), _p(om), int(n))
    return om.reshape(cfg.ny, cfg.nx)


def mesh_jacobi(cfg, om, x, mu):
    """mu Jacobi sweeps of the Sec. 5 mesh equations with om [ny][nx] frozen,
    from x [2][ny][nx]; returns X^[mu]."""
    N = cfg.nx * cfg.ny
    X = np.zeros(2 * N)
    lib().oref_jacobi(ctypes.byref(cfg), _p(_vec(om, N)), _p(_vec(x, 2 * N)), int(mu), _p(X))
    return X.reshape(2, cfg.ny, cfg.nx)


def mesh(cfg, cons, J, x, dt=0.0):
    """Mesh velocity, limiter value and step: (xdot, dtau, dt).  dt <= 0 selects
    the CFL step with the mesh motion included."""
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    xdot = np.zeros(2 * N)
    tau, dto = np.zeros(1), np.zeros(1)
    st = lib().oref_mesh(ctypes.byref(cfg), _p(_vec(cons, nv * N)), _p(_vec(J, N)),
                         _p(_vec(x, 2 * N)), float(dt), _p(xdot), _p(tau), _p(dto))
    if st != 0:
        raise RuntimeError("oracle mesh: cons2prim failed")
    return xdot.reshape(2, cfg.ny, cfg.nx), tau[0], dto[0]


def rk_step(cfg, cons, J, x, dt=0.0):
    """One SSP-RK3 step; returns new (cons, J, x, dt_used)."""
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    cons = _vec(cons, nv * N).copy()
    J = _vec(J, N).copy()
    x = _vec(x, 2 * N).copy()
    dtu = np.zeros(1)
    st = lib().oref_rk_step(ctypes.byref(cfg), _p(cons), _p(J), _p(x), float(dt), _p(dtu))
    if st != 0:
        raise RuntimeError("oracle rk_step: cons2prim failed")
    return (cons.reshape(nv, cfg.ny, cfg.nx), J.reshape(cfg.ny, cfg.nx),
            x.reshape(2, cfg.ny, cfg.nx), dtu[0])


def rk_step_given(cfg, cons, J, x, xdot, dt):
    """One SSP-RK3 step with a given mesh velocity and step."""
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    cons = _vec(cons, nv * N).copy()
    J = _vec(J, N).copy()
    x = _vec(x, 2 * N).copy()
    st = lib().oref_rk_step_given(ctypes.byref(cfg), _p(cons), _p(J), _p(x), _p(_vec(xdot, 2 * N)), float(dt))
    if st != 0:
        raise RuntimeError("oracle rk_step_given: cons2prim failed")
    return cons.reshape(nv, cfg.ny, cfg.nx), J.reshape(cfg.ny, cfg.nx), x.reshape(2, cfg.ny, cfg.nx)


def totals(cfg, cons, J, dcons=None, dJ=None):
    N = cfg.nx * cfg.ny
    nv = nvar(cfg)
    out = np.zeros(4)
    dc = _vec(dcons, nv * N) if dcons is not None else None
    dj = _vec(dJ, N) if dJ is not None else None
    lib().oref_totals(ctypes.byref(cfg), _p(_vec(cons, nv * N)), _p(_vec(J, N)), _p(dc), _p(dj),
                      _p(out))
    return out


# ---- RMHD pointwise functions (8-component states) ---------------------------
def mhd_prim2cons(gamma, w):
    U = np.zeros(8)
    lib().oref_mhd_prim2cons(gamma, _p(_vec(w, 8)), _p(U))
    return U


def mhd_cons2prim(gamma, U):
    w = np.zeros(8)
    it = ctypes.c_int(0)
    st = lib().oref_mhd_cons2prim(gamma, _p(_vec(U, 8)), _p(w), ctypes.byref(it))
    return w, st, it.value


def mhd_flux(gamma, w, direction):
    F = np.zeros(8)
    lib().oref_mhd_flux(gamma, _p(_vec(w, 8)), direction, _p(F))
    return F


def mhd_entropy(gamma, w):
    return lib().oref_mhd_entropy(gamma, _p(_vec(w, 8)))


def mhd_entropy_vars(gamma, w):
    V = np.zeros(8)
    lib().oref_mhd_entropy_vars(gamma, _p(_vec(w, 8)), _p(V))
    return V


def mhd_potentials(w):
    """(phi, psi[3], Phi)."""
    phi, psi, Phi = np.zeros(1), np.zeros(3), np.zeros(1)
    lib().oref_mhd_potentials(_p(_vec(w, 8)), _p(phi), _p(psi), _p(Phi))
    return phi[0], psi, Phi[0]


def mhd_phiprime(w):
    P = np.zeros(8)
    lib().oref_mhd_phiprime(_p(_vec(w, 8)), _p(P))
    return P


def mhd_ec_flux(gamma, wl, wr):
    """(U~[8], F~[3][8])."""
    Ut, Ft = np.zeros(8), np.zeros(24)
    lib().oref_mhd_ec_flux(gamma, _p(_vec(wl, 8)), _p(_vec(wr, 8)), _p(Ut), _p(Ft))
    return Ut, Ft.reshape(3, 8)


def mhd_eigen(gamma, w_rot):
    lam, R = np.zeros(8), np.zeros(64)
    lib().oref_mhd_eigen(gamma, _p(_vec(w_rot, 8)), _p(lam), _p(R))
    return lam, R.reshape(8, 8)


# ---- 3D RMHD grid functions --------------------------------------------------
def make_cfg3(nx, ny, nz, bc=(PERIODIC, PERIODIC, PERIODIC), period=(1.0, 1.0, 1.0), gamma=4.0 / 3.0,
              p=2, w=5, weno_eps=1e-6, cfl=0.3, monitor=MONITOR_LNRHO, alpha=800.0, n_filter=4, mu=10,
              move_mesh=1, alpha_lap=0.0, inflow=None) -> Cfg3:
    c = Cfg3()
    c.nx, c.ny, c.nz = nx, ny, nz
    for k in range(3):
        c.bc[k] = bc[k]
        c.period[k] = period[k]
    c.gamma, c.p, c.w, c.weno_eps, c.cfl = gamma, p, w, weno_eps, cfl
    c.monitor, c.alpha, c.n_filter, c.mu, c.move_mesh = monitor, alpha, n_filter, mu, move_mesh
    c.alpha_lap = alpha_lap
    for a, v in enumerate(inflow if inflow is not None else ()):
        c.inflow[a] = v
    return c


def _shape3(cfg, ncomp):
    return (ncomp, cfg.nz, cfg.ny, cfg.nx) if ncomp > 1 else (cfg.nz, cfg.ny, cfg.nx)


def metrics3(cfg, x):
    N = cfg.nx * cfg.ny * cfg.nz
    m, J0 = np.zeros(9 * N), np.zeros(N)
    lib().oref3_metrics(ctypes.byref(cfg), _p(_vec(x, 3 * N)), _p(m), _p(J0))
    return m.reshape(_shape3(cfg, 9)), J0.reshape(_shape3(cfg, 1))


def init_state3(cfg, prim, x):
    N = cfg.nx * cfg.ny * cfg.nz
    cons, J = np.zeros(8 * N), np.zeros(N)
    lib().oref3_init_state(ctypes.byref(cfg), _p(_vec(prim, 8 * N)), _p(_vec(x, 3 * N)), _p(cons), _p(J))
    return cons.reshape(_shape3(cfg, 8)), J.reshape(_shape3(cfg, 1))


def state_prim3(cfg, cons, J):
    N = cfg.nx * cfg.ny * cfg.nz
    prim = np.zeros(8 * N)
    st = lib().oref3_state_prim(ctypes.byref(cfg), _p(_vec(cons, 8 * N)), _p(_vec(J, N)), _p(prim))
    return prim.reshape(_shape3(cfg, 8)), st


def rhs3(cfg, cons, J, x, xdot=None):
    N = cfg.nx * cfg.ny * cfg.nz
    if xdot is None:
        xdot = np.zeros(3 * N)
    dcons, dJ = np.zeros(8 * N), np.zeros(N)
    st = lib().oref3_rhs(ctypes.byref(cfg), _p(_vec(cons, 8 * N)), _p(_vec(J, N)), _p(_vec(x, 3 * N)),
                         _p(_vec(xdot, 3 * N)), _p(dcons), _p(dJ))
    if st != 0:
        raise RuntimeError("oracle rhs3: cons2prim failed")
    return dcons.reshape(_shape3(cfg, 8)), dJ.reshape(_shape3(cfg, 1))


def cfl_dt3(cfg, cons, J, x):
    N = cfg.nx * cfg.ny * cfg.nz
    dt = np.zeros(1)
    st = lib().oref3_cfl_dt(ctypes.byref(cfg), _p(_vec(cons, 8 * N)), _p(_vec(J, N)), _p(_vec(x, 3 * N)), _p(dt))
    if st != 0:
        raise RuntimeError("oracle cfl3: cons2prim failed")
    return dt[0]


def monitor3(cfg, cons, J):
    """:func:`monitor` in 3D ([nz][ny][nx])."""
    N = cfg.nx * cfg.ny * cfg.nz
    om = np.zeros(N)
    st = lib().oref3_monitor(ctypes.byref(cfg), _p(_vec(cons, 8 * N)), _p(_vec(J, N)), _p(om))
    if st != 0:
        raise RuntimeError("oracle monitor3: cons2prim failed")
    return om.reshape(cfg.nz, cfg.ny, cfg.nx)


def mesh_filter3(cfg, om, n):
    """:func:`mesh_filter` in 3D ([nz][ny][nx])."""
    N = cfg.nx * cfg.ny * cfg.nz
    om = _vec(om, N).copy()
    lib().oref3_filter(ctypes.byref(cfg), _p(om), int(n))
    return om.reshape(cfg.nz, cfg.ny, cfg.nx)


def mesh_jacobi3(cfg, om, x, mu):
    """:func:`mesh_jacobi` in 3D: x [3][nz][ny][nx]."""
    N = cfg.nx * cfg.ny * cfg.nz
    X = np.zeros(3 * N)
    lib().oref3_jacobi(ctypes.byref(cfg), _p(_vec(om, N)), _p(_vec(x, 3 * N)), int(mu), _p(X))
    return X.reshape(_shape3(cfg, 3))


def mesh3(cfg, cons, J, x, dt=0.0):
    """(xdot, dtau, dt) as :func:`mesh`, in 3D."""
    N = cfg.nx * cfg.ny * cfg.nz
    xdot, tau, dto = np.zeros(3 * N), np.zeros(1), np.zeros(1)
    st = lib().oref3_mesh(ctypes.byref(cfg), _p(_vec(cons, 8 * N)), _p(_vec(J, N)), _p(_vec(x, 3 * N)),
                          float(dt), _p(xdot), _p(tau), _p(dto))
    if st != 0:
        raise RuntimeError("oracle mesh3: cons2prim failed")
    return xdot.reshape(_shape3(cfg, 3)), tau[0], dto[0]


def rk_step3(cfg, cons, J, x, dt=0.0):
    N = cfg.nx * cfg.ny * cfg.nz
    cons, J, x = _vec(cons, 8 * N).copy(), _vec(J, N).copy(), _vec(x, 3 * N).copy()
    dtu = np.zeros(1)
    st = lib().oref3_rk_step(ctypes.byref(cfg), _p(cons), _p(J), _p(x), float(dt), _p(dtu))
    if st != 0:
        raise RuntimeError("oracle rk_step3: cons2prim failed")
    return cons.reshape(_shape3(cfg, 8)), J.reshape(_shape3(cfg, 1)), x.reshape(_shape3(cfg, 3)), dtu[0]


def rk_step3_given(cfg, cons, J, x, xdot, dt):
    """One 3D SSP-RK3 step with a given mesh velocity [3][nz][ny][nx] and step."""
    N = cfg.nx * cfg.ny * cfg.nz
    cons, J, x = _vec(cons, 8 * N).copy(), _vec(J, N).copy(), _vec(x, 3 * N).copy()
    st = lib().oref3_rk_step_given(ctypes.byref(cfg), _p(cons), _p(J), _p(x), _p(_vec(xdot, 3 * N)), float(dt))
    if st != 0:
        raise RuntimeError("oracle rk_step3_given: cons2prim failed")
    return cons.reshape(_shape3(cfg, 8)), J.reshape(_shape3(cfg, 1)), x.reshape(_shape3(cfg, 3))


def totals3(cfg, cons, J, dcons=None, dJ=None):
    N = cfg.nx * cfg.ny * cfg.nz
    out = np.zeros(4)
    dc = _vec(dcons, 8 * N) if dcons is not None else None
    dj = _vec(dJ, N) if dJ is not None else None
    lib().oref3_totals(ctypes.byref(cfg), _p(_vec(cons, 8 * N)), _p(_vec(J, N)), _p(dc), _p(dj), _p(out))
    return out
