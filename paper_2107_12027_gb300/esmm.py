"""Thin ctypes binding of libesmm (the C ABI of ``include/esmm.h``).

Argument marshalling only: every step of the scheme runs in the CUDA library.
Arrays may be numpy arrays (host memory, ``ESMM_MEM_HOST``) or CUDA torch
tensors (device memory, ``ESMM_MEM_DEVICE``); they must be C-contiguous FP64
with the layouts of the header.  The library must have been built
(``paper_2107_12027_gb300.build.build()``); importing this module without it,
or calling into it without a GPU, raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_CUDA, ERR_C2P, ERR_TIMEOUT, ERR_STATE = 0, 1, 2, 3, 4, 5
RHD, RMHD = 0, 1
PERIODIC, OUTFLOW, INFLOW = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
FP64, MIXED = 0, 1
SWEEP_AUTO, SWEEP_FUSED, SWEEP_SPLIT = 0, 1, 2
MONITOR_RHO, MONITOR_LNRHO = 0, 1
GET_PRIM, GET_CONS, GET_J, GET_X, GET_XDOT = 0, 1, 2, 3, 4
_ERR = {1: "ESMM_ERR_ARG", 2: "ESMM_ERR_CUDA", 3: "ESMM_ERR_C2P", 4: "ESMM_ERR_TIMEOUT", 5: "ESMM_ERR_STATE"}

#: The paper's named schemes (Sec. 6): EC flux order 2p, WENO order w of the
#: ES dissipation (0: the EC scheme alone) and whether the mesh adapts.
SCHEMES = {
    "MM-O6": dict(p=3, w=0, move_mesh=1),   # sixth-order EC on the moving mesh
    "MM-O5": dict(p=3, w=5, move_mesh=1),   # fifth-order ES, adaptive moving mesh
    "UM-O6": dict(p=3, w=0, move_mesh=0),   # the EC scheme on the static mesh
    "UM-O5": dict(p=3, w=5, move_mesh=0),   # the ES scheme on the static mesh
}


def _apply_scheme(scheme, p, w, params):
    """(p, w) of a named scheme (or the given ones), with its mesh switch put
    into params unless the caller set move_mesh."""
    if scheme is None:
        return p, w
    s = SCHEMES[scheme]
    params.setdefault("move_mesh", s["move_mesh"])
    return s["p"], s["w"]


#: every entry point declared in include/esmm.h
SYMBOLS = (
    "esmm_grid_create", "esmm_grid_destroy", "esmm_set_stream", "esmm_set_eos", "esmm_set_order",
    "esmm_set_params", "esmm_get_params", "esmm_state_set", "esmm_state_set_cons", "esmm_state_get",
    "esmm_get_time", "esmm_rhs", "esmm_cfl_dt", "esmm_mesh_redistribute", "esmm_rk_step", "esmm_rk_step_given",
    "esmm_set_inflow",
    "esmm_advance", "esmm_totals", "esmm_last_error", "esmm_version", "esmm_profile", "esmm_profile_read",
    "esmm_rhs_static", "esmm_fma_peak", "esmm_flux_ops", "esmm_mhd_eigen", "esmm_batch_create", "esmm_batch_size", "esmm_batch_state_set", "esmm_batch_state_get",
    "esmm_batch_times", "esmm_batch_totals", "esmm_tune", "esmm_adjoint_record", "esmm_adjoint_steps",
    "esmm_adjoint_checkpoint", "esmm_adjoint_replay", "esmm_adjoint_vjp", "esmm_rhs_vjp",
    "esmm_slab_create", "esmm_slab_rows",
)
SLAB_HALO = 16
TUNE_SLOTS = 17
OP_MAX, OP_MIN, OP_SUM = 0, 1, 2
_dptr = ctypes.POINTER(ctypes.c_double)
#: comm callbacks of esmm_slab_create (include/esmm.h esmm_comm)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, _dptr, ctypes.c_int, ctypes.c_int)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, _dptr, _dptr, _dptr, _dptr, ctypes.c_longlong)


class Comm(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("allreduce", ALLREDUCE_FN), ("exchange", EXCHANGE_FN)]
STATIC_MAX_PADDED_NODES = 68644
KIND_NODE, KIND_PAIRS, KIND_IFACE, KIND_UPDATE, KIND_MESH, KIND_OTHER = range(6)
KINDS = ("node", "pairs", "iface", "update", "mesh", "other")


class Params(ctypes.Structure):
    _fields_ = [("cfl", ctypes.c_double), ("weno_eps", ctypes.c_double), ("monitor", ctypes.c_int),
                ("alpha", ctypes.c_double), ("n_filter", ctypes.c_int), ("mu", ctypes.c_int),
                ("move_mesh", ctypes.c_int), ("precision", ctypes.c_int),
                ("alpha_lap", ctypes.c_double), ("sweep", ctypes.c_int)]


_lib = None


class EsmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERR.get(code, code), msg))
        self.code = code


def lib():
    """Load libesmm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libesmm.so is not built (%s); run paper_2107_12027_gb300.build.build()" % _build.LIB)
        L = ctypes.CDLL(_build.LIB)
        vp, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "esmm_grid_create": [ctypes.POINTER(vp), i, ctypes.POINTER(i), dp, dp, i, ctypes.POINTER(i), vp],
            "esmm_grid_destroy": [vp], "esmm_set_stream": [vp, vp], "esmm_set_eos": [vp, d],
            "esmm_set_order": [vp, i, i], "esmm_set_params": [vp, ctypes.POINTER(Params)],
            "esmm_get_params": [vp, ctypes.POINTER(Params)], "esmm_state_set": [vp, vp, vp, i],
            "esmm_state_set_cons": [vp, vp, vp, vp, d, i], "esmm_state_get": [vp, i, vp, i],
            "esmm_get_time": [vp, dp], "esmm_rhs": [vp, vp, vp, vp, vp, vp, vp, i],
            "esmm_cfl_dt": [vp, dp], "esmm_mesh_redistribute": [vp, d, vp, dp, dp, i],
            "esmm_rk_step": [vp, d, dp], "esmm_rk_step_given": [vp, vp, d, i], "esmm_set_inflow": [vp, dp], "esmm_advance": [vp, i, d], "esmm_totals": [vp, dp],
            "esmm_last_error": [vp, ctypes.POINTER(i), ctypes.c_char_p, i],
            "esmm_profile": [vp, i],
            "esmm_rhs_static": [i, i, ctypes.POINTER(i), dp, dp, d, i, i, vp, vp, vp, vp, vp, vp, vp],
            "esmm_mhd_eigen": [d, i, vp, vp, vp, vp, vp, vp],
            "esmm_fma_peak": [i, d, dp, dp],
            "esmm_flux_ops": [d, i, i, dp],
            "esmm_batch_create": [ctypes.POINTER(vp), i, ctypes.POINTER(i), dp, dp, ctypes.POINTER(i), i, vp],
            "esmm_batch_size": [vp, ctypes.POINTER(i)],
            "esmm_batch_state_set": [vp, i, vp, vp, i],
            "esmm_batch_state_get": [vp, i, i, vp, i],
            "esmm_batch_times": [vp, dp], "esmm_batch_totals": [vp, dp],
            "esmm_tune": [vp, ctypes.POINTER(i)],
            "esmm_adjoint_record": [vp, i, d], "esmm_adjoint_steps": [vp, ctypes.POINTER(i), dp],
            "esmm_adjoint_checkpoint": [vp, i, i, vp, i], "esmm_adjoint_replay": [vp, i],
            "esmm_adjoint_vjp": [vp, vp, vp, vp, i], "esmm_rhs_vjp": [vp, vp, vp, vp, vp, vp, vp, i],
            "esmm_profile_read": [vp, dp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)],
            "esmm_slab_create": [ctypes.POINTER(vp), ctypes.POINTER(i), dp, dp, i, ctypes.POINTER(i), i, i,
                                 ctypes.POINTER(Comm), vp],
            "esmm_slab_rows": [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.esmm_version.restype = ctypes.c_char_p
        L.esmm_version.argtypes = []
        _lib = L
    return _lib


def version() -> str:
    return lib().esmm_version().decode()


def mhd_eigen(gamma, w, dw=None):
    """Scaled RMHD eigen-system of rotated primitive states w [n][8] (and, with
    dw, its tangent): (lam [n][8], R [n][8][8]) or (lam, R, dlam, dR)."""
    w = np.ascontiguousarray(np.atleast_2d(w), dtype=np.float64)
    n = w.shape[0]
    lam, R = np.empty((n, 8)), np.empty((n, 8, 8))
    args = [float(gamma), n, w.ctypes.data, None, lam.ctypes.data, R.ctypes.data, None, None]
    if dw is not None:
        dw = np.ascontiguousarray(np.atleast_2d(dw), dtype=np.float64)
        dlam, dR = np.empty((n, 8)), np.empty((n, 8, 8))
        args[3], args[6], args[7] = dw.ctypes.data, dlam.ctypes.data, dR.ctypes.data
    rc = lib().esmm_mhd_eigen(*args)
    if rc != OK:
        raise EsmmError(rc, "esmm_mhd_eigen")
    return (lam, R) if dw is None else (lam, R, dlam, dR)


def fma_peak(precision, seconds=1.0):
    """esmm_fma_peak: measured FMA throughput (flop/s, ms per launch) of the
    FP64 (precision FP64) or FP32 (precision MIXED) pipe."""
    fl, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib().esmm_fma_peak(int(precision), float(seconds), ctypes.byref(fl), ctypes.byref(ms))
    if rc != OK:
        raise EsmmError(rc, "esmm_fma_peak")
    return fl.value, ms.value


def flux_ops(gamma, p, w):
    """esmm_flux_ops: algorithmic operations of one two-point flux, of one
    interface's ES dissipation and of the interface kernel's combination."""
    ops = (ctypes.c_double * 3)()
    rc = lib().esmm_flux_ops(float(gamma), int(p), int(w), ops)
    if rc != OK:
        raise EsmmError(rc, "esmm_flux_ops")
    return {"pair": ops[0], "dissipation": ops[1], "combination": ops[2]}


def rhs_static(nx, ny, bc, lo, hi, gamma, p, w, cons, J, x, xdot, dcons, dJ, stream=None):
    """esmm_rhs_static: the allocation-free right-hand side (device tensors only).

    Enqueues on ``stream`` (a raw cudaStream_t handle, None for the legacy
    default stream) and returns the status code."""
    ptrs = [_ptr(a) for a in (cons, J, x, dcons, dJ)]
    assert all(m == MEM_DEVICE for _, m in ptrs), "esmm_rhs_static takes device tensors"
    xd = _ptr(xdot)[0] if xdot is not None else None
    b = (ctypes.c_int * 2)(bc[0], bc[1])
    l2 = (ctypes.c_double * 2)(lo[0], lo[1])
    h2 = (ctypes.c_double * 2)(hi[0], hi[1])
    st = ctypes.c_void_p(stream) if stream is not None else None
    return lib().esmm_rhs_static(int(nx), int(ny), b, l2, h2, float(gamma), int(p), int(w), ptrs[0][0],
                                 ptrs[1][0], ptrs[2][0], xd, ptrs[3][0], ptrs[4][0], st)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, n=None):
    """(pointer, mem) of a numpy array or CUDA torch tensor (FP64, contiguous)."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch
        assert a.dtype == torch.float64 and a.is_cuda and a.is_contiguous(), "need a contiguous CUDA float64 tensor"
        assert n is None or a.numel() == n
        return ctypes.c_void_p(a.data_ptr()), MEM_DEVICE
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], \
        "need a C-contiguous float64 numpy array"
    assert n is None or a.size == n
    return ctypes.c_void_p(a.ctypes.data), MEM_HOST


def _mem(*arrays):
    mems = {m for _, m in arrays if m is not None}
    assert len(mems) == 1, "arrays must all be host (numpy) or all device (torch)"
    return mems.pop()


class Grid:
    """One 2D problem (RHD: 4 unknowns per node, RMHD: 8): a handle of the C
    ABI plus argument marshalling."""

    def __init__(self, n, lo=(0.0, 0.0), hi=(1.0, 1.0), bc=(PERIODIC, PERIODIC), gamma=5.0 / 3.0, p=2, w=5,
                 stream=None, phys=RHD, scheme=None, **params):
        p, w = _apply_scheme(scheme, p, w, params)
        self.nx, self.ny = int(n[0]), int(n[1])
        self.N = self.nx * self.ny
        self.phys = phys
        self.nv = 8 if phys == RMHD else 4
        h = ctypes.c_void_p()
        nn = (ctypes.c_int * 3)(self.nx, self.ny, 1)
        lo3 = (ctypes.c_double * 3)(lo[0], lo[1], 0.0)
        hi3 = (ctypes.c_double * 3)(hi[0], hi[1], 1.0)
        bc3 = (ctypes.c_int * 3)(bc[0], bc[1], 0)
        st = ctypes.c_void_p(stream) if stream is not None else None
        self._check(lib().esmm_grid_create(ctypes.byref(h), 2, nn, lo3, hi3, phys, bc3, st))
        self.h = h
        self.set_eos(gamma)
        self.set_order(p, w)
        if params:
            self.set_params(**params)

    # -- plumbing -----------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            msg = ""
            h = getattr(self, "h", None)
            if h is not None:
                buf = ctypes.create_string_buffer(256)
                lib().esmm_last_error(h, None, buf, 256)
                msg = buf.value.decode()
            raise EsmmError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "h", None) is not None:
            lib().esmm_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- configuration -------------------------------------------------------
    def set_stream(self, stream):
        self._check(lib().esmm_set_stream(self.h, ctypes.c_void_p(stream)))

    def set_eos(self, gamma):
        self._check(lib().esmm_set_eos(self.h, float(gamma)))

    def set_order(self, p, w):
        self._check(lib().esmm_set_order(self.h, int(p), int(w)))

    def get_params(self):
        prm = Params()
        self._check(lib().esmm_get_params(self.h, ctypes.byref(prm)))
        return {k: getattr(prm, k) for k, _ in Params._fields_}

    def set_inflow(self, prim):
        """The primitive state held beyond every INFLOW end (nv values)."""
        a = (ctypes.c_double * self.nv)(*[float(v) for v in prim])
        self._check(lib().esmm_set_inflow(self.h, a))

    def set_params(self, **kw):
        cur = self.get_params()
        cur.update(kw)
        prm = Params(**cur)
        self._check(lib().esmm_set_params(self.h, ctypes.byref(prm)))

    # -- state ----------------------------------------------------------------
    def state_set(self, prim, x=None):
        pp, mp = _ptr(prim, self.nv * self.N)
        px, mx = _ptr(x, 2 * self.N)
        self._check(lib().esmm_state_set(self.h, pp, px, _mem((pp, mp), (px, mx))))

    def state_set_cons(self, cons, J, x, t=0.0):
        a = [_ptr(cons, self.nv * self.N), _ptr(J, self.N), _ptr(x, 2 * self.N)]
        self._check(lib().esmm_state_set_cons(self.h, a[0][0], a[1][0], a[2][0], float(t), _mem(*a)))

    def state_get(self, what, out=None):
        size = {GET_PRIM: self.nv, GET_CONS: self.nv, GET_J: 1, GET_X: 2, GET_XDOT: 2}[what]
        shape = (size, self.ny, self.nx) if size > 1 else (self.ny, self.nx)
        if out is None:
            out = np.empty(shape)
        po, mo = _ptr(out, size * self.N)
        self._check(lib().esmm_state_get(self.h, what, po, mo))
        return out

    def time(self):
        t = ctypes.c_double()
        self._check(lib().esmm_get_time(self.h, ctypes.byref(t)))
        return t.value

    # -- the scheme -----------------------------------------------------------
    def rhs(self, cons, J, x, xdot=None, dcons=None, dJ=None):
        """d(cons)/dt, dJ/dt of the semi-discrete ES scheme (host or device)."""
        host = not _is_torch(cons)
        if dcons is None:
            if host:
                dcons, dJ = np.empty((self.nv, self.ny, self.nx)), np.empty((self.ny, self.nx))
            else:
                import torch
                dcons = torch.empty((self.nv, self.ny, self.nx), dtype=torch.float64, device=cons.device)
                dJ = torch.empty((self.ny, self.nx), dtype=torch.float64, device=cons.device)
        a = [_ptr(cons, self.nv * self.N), _ptr(J, self.N), _ptr(x, 2 * self.N)]
        xd = _ptr(xdot, 2 * self.N)
        o = [_ptr(dcons, self.nv * self.N), _ptr(dJ, self.N)]
        mem = _mem(*a, *o, *([xd] if xdot is not None else []))
        self._check(lib().esmm_rhs(self.h, a[0][0], a[1][0], a[2][0], xd[0], o[0][0], o[1][0], mem))
        return dcons, dJ

    def cfl_dt(self):
        dt = ctypes.c_double()
        self._check(lib().esmm_cfl_dt(self.h, ctypes.byref(dt)))
        return dt.value

    def mesh_redistribute(self, dt=0.0):
        """(xdot, dtau, dt): the mesh velocity, limiter value and step
        (dt <= 0: the CFL step with the mesh motion included)."""
        xdot = np.empty((2, self.ny, self.nx))
        tau, dtu = ctypes.c_double(), ctypes.c_double()
        self._check(lib().esmm_mesh_redistribute(self.h, float(dt), ctypes.c_void_p(xdot.ctypes.data),
                                                  ctypes.byref(tau), ctypes.byref(dtu), MEM_HOST))
        return xdot, tau.value, dtu.value

    def rk_step(self, dt=0.0, sync=True):
        """One SSP-RK3 step; returns the step used when sync (else None)."""
        if sync:
            d = ctypes.c_double()
            self._check(lib().esmm_rk_step(self.h, float(dt), ctypes.byref(d)))
            return d.value
        self._check(lib().esmm_rk_step(self.h, float(dt), None))
        return None

    def rk_step_given(self, xdot, dt):
        """One step with the prescribed mesh velocity xdot ([d][...], numpy or
        CUDA tensor, d = 2 or 3) held over the step; dt > 0."""
        nd = 3 if isinstance(self, Grid3) else 2
        px, mx = _ptr(xdot, nd * self.N)
        self._check(lib().esmm_rk_step_given(self.h, px, float(dt), mx))

    def advance(self, nsteps, dt=0.0):
        self._check(lib().esmm_advance(self.h, int(nsteps), float(dt)))

    def totals(self):
        out = (ctypes.c_double * 3)()
        self._check(lib().esmm_totals(self.h, out))
        return np.array(out[:])

    def profile(self, mask=0):
        """Reset the launch counters; time the kernel kinds in mask (bit k = kind k)."""
        self._check(lib().esmm_profile(self.h, int(mask)))

    def profile_read(self):
        """{kind: (device ms of timed launches, launches, timed launches)}."""
        ms = (ctypes.c_double * 6)()
        n = (ctypes.c_longlong * 6)()
        t = (ctypes.c_longlong * 6)()
        self._check(lib().esmm_profile_read(self.h, ms, n, t))
        return {KINDS[k]: (ms[k], n[k], t[k]) for k in range(6)}

    # -- adjoint ------------------------------------------------------------
    def adjoint_record(self, nsteps, dt=0.0):
        """Advance nsteps steps keeping per-step checkpoints for the adjoint."""
        self._check(lib().esmm_adjoint_record(self.h, int(nsteps), float(dt)))

    def adjoint_steps(self):
        n = ctypes.c_int()
        self._check(lib().esmm_adjoint_steps(self.h, ctypes.byref(n), None))
        dts = (ctypes.c_double * max(n.value, 1))()
        self._check(lib().esmm_adjoint_steps(self.h, ctypes.byref(n), dts))
        return np.array(dts[:n.value])

    def adjoint_checkpoint(self, step, what, out=None):
        size = {GET_CONS: self.nv, GET_J: 1, GET_X: 2, GET_XDOT: 2}[what]
        if out is None:
            out = np.empty((size, self.ny, self.nx) if size > 1 else (self.ny, self.nx))
        po, mo = _ptr(out, size * self.N)
        self._check(lib().esmm_adjoint_checkpoint(self.h, int(step), what, po, mo))
        return out

    def adjoint_replay(self, nsteps):
        """Re-run the recorded map (recorded mesh velocities and steps) from
        the current state."""
        self._check(lib().esmm_adjoint_replay(self.h, int(nsteps)))

    def adjoint_vjp(self, lam_final, lam_cons0=None, lam_prim0=None):
        """dF/d(cons^0) and dF/d(prim^0) from lam_final = dF/d(cons^final)."""
        host = not _is_torch(lam_final)
        if host:
            lam_cons0 = np.empty((self.nv, self.ny, self.nx)) if lam_cons0 is None else lam_cons0
            lam_prim0 = np.empty((self.nv, self.ny, self.nx)) if lam_prim0 is None else lam_prim0
        a = _ptr(lam_final, self.nv * self.N)
        c = _ptr(lam_cons0, self.nv * self.N)
        p_ = _ptr(lam_prim0, self.nv * self.N)
        mem = _mem(a, *([c] if lam_cons0 is not None else []), *([p_] if lam_prim0 is not None else []))
        self._check(lib().esmm_adjoint_vjp(self.h, a[0], c[0], p_[0], mem))
        return lam_cons0, lam_prim0

    def rhs_vjp(self, cons, J, x, xdot, mu, lam=None):
        """(d rhs / d cons)^T mu at (cons, J, x, xdot) with J, x, xdot fixed."""
        if lam is None:
            lam = np.empty((self.nv, self.ny, self.nx))
        a = [_ptr(cons, self.nv * self.N), _ptr(J, self.N), _ptr(x, 2 * self.N), _ptr(mu, self.nv * self.N),
             _ptr(lam, self.nv * self.N)]
        xd = _ptr(xdot, 2 * self.N)
        mem = _mem(*a, *([xd] if xdot is not None else []))
        self._check(lib().esmm_rhs_vjp(self.h, a[0][0], a[1][0], a[2][0], xd[0], a[3][0], a[4][0], mem))
        return lam

    def tune(self):
        """Run the launch autotuner on the current state; returns the 13 chosen
        block sizes (negative: largest problem first) and the 4 tile shapes of
        the pair and interface launches (tx, + 1000 for a persistent grid)."""
        bs = (ctypes.c_int * TUNE_SLOTS)()
        self._check(lib().esmm_tune(self.h, bs))
        return list(bs)

    def last_error(self):
        n = ctypes.c_int()
        buf = ctypes.create_string_buffer(256)
        self._check(lib().esmm_last_error(self.h, ctypes.byref(n), buf, 256))
        return n.value, buf.value.decode()


class Grid3(Grid):
    """One 3D RMHD problem (n = (nx, ny, nz)); arrays are [c][z][y][x] with 8
    state components and 3 mesh components."""

    def __init__(self, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(PERIODIC, PERIODIC, PERIODIC),
                 gamma=4.0 / 3.0, p=2, w=5, stream=None, scheme=None, **params):
        p, w = _apply_scheme(scheme, p, w, params)
        self.nx, self.ny, self.nz = int(n[0]), int(n[1]), int(n[2])
        self.N = self.nx * self.ny * self.nz
        self.phys, self.nv = RMHD, 8
        h = ctypes.c_void_p()
        nn = (ctypes.c_int * 3)(self.nx, self.ny, self.nz)
        lo3 = (ctypes.c_double * 3)(*lo)
        hi3 = (ctypes.c_double * 3)(*hi)
        bc3 = (ctypes.c_int * 3)(*bc)
        st = ctypes.c_void_p(stream) if stream is not None else None
        self._check(lib().esmm_grid_create(ctypes.byref(h), 3, nn, lo3, hi3, RMHD, bc3, st))
        self.h = h
        self.set_eos(gamma)
        self.set_order(p, w)
        if params:
            self.set_params(**params)

    def _shape(self, c):
        return (c, self.nz, self.ny, self.nx) if c > 1 else (self.nz, self.ny, self.nx)

    def state_set(self, prim, x=None):
        pp, mp = _ptr(prim, 8 * self.N)
        px, mx = _ptr(x, 3 * self.N)
        self._check(lib().esmm_state_set(self.h, pp, px, _mem((pp, mp), (px, mx))))

    def state_set_cons(self, cons, J, x, t=0.0):
        a = [_ptr(cons, 8 * self.N), _ptr(J, self.N), _ptr(x, 3 * self.N)]
        self._check(lib().esmm_state_set_cons(self.h, a[0][0], a[1][0], a[2][0], float(t), _mem(*a)))

    def state_get(self, what, out=None):
        size = {GET_PRIM: 8, GET_CONS: 8, GET_J: 1, GET_X: 3, GET_XDOT: 3}[what]
        if out is None:
            out = np.empty(self._shape(size))
        po, mo = _ptr(out, size * self.N)
        self._check(lib().esmm_state_get(self.h, what, po, mo))
        return out

    def rhs(self, cons, J, x, xdot=None, dcons=None, dJ=None):
        host = not _is_torch(cons)
        if dcons is None:
            if host:
                dcons, dJ = np.empty(self._shape(8)), np.empty(self._shape(1))
            else:
                import torch
                dcons = torch.empty(self._shape(8), dtype=torch.float64, device=cons.device)
                dJ = torch.empty(self._shape(1), dtype=torch.float64, device=cons.device)
        a = [_ptr(cons, 8 * self.N), _ptr(J, self.N), _ptr(x, 3 * self.N)]
        xd = _ptr(xdot, 3 * self.N)
        o = [_ptr(dcons, 8 * self.N), _ptr(dJ, self.N)]
        mem = _mem(*a, *o, *([xd] if xdot is not None else []))
        self._check(lib().esmm_rhs(self.h, a[0][0], a[1][0], a[2][0], xd[0], o[0][0], o[1][0], mem))
        return dcons, dJ

    def adjoint_checkpoint(self, step, what, out=None):
        size = {GET_CONS: 8, GET_J: 1, GET_X: 3, GET_XDOT: 3}[what]
        if out is None:
            out = np.empty(self._shape(size))
        po, mo = _ptr(out, size * self.N)
        self._check(lib().esmm_adjoint_checkpoint(self.h, int(step), what, po, mo))
        return out

    def adjoint_vjp(self, lam_final, lam_cons0=None, lam_prim0=None):
        """dF/d(cons^0) and dF/d(prim^0) from lam_final = dF/d(cons^final)."""
        if not _is_torch(lam_final):
            lam_cons0 = np.empty(self._shape(8)) if lam_cons0 is None else lam_cons0
            lam_prim0 = np.empty(self._shape(8)) if lam_prim0 is None else lam_prim0
        a = _ptr(lam_final, 8 * self.N)
        c = _ptr(lam_cons0, 8 * self.N)
        p_ = _ptr(lam_prim0, 8 * self.N)
        mem = _mem(a, *([c] if lam_cons0 is not None else []), *([p_] if lam_prim0 is not None else []))
        self._check(lib().esmm_adjoint_vjp(self.h, a[0], c[0], p_[0], mem))
        return lam_cons0, lam_prim0

    def rhs_vjp(self, cons, J, x, xdot, mu, lam=None):
        """(d rhs / d cons)^T mu at (cons, J, x, xdot) with J, x, xdot fixed."""
        if lam is None:
            lam = np.empty(self._shape(8))
        a = [_ptr(cons, 8 * self.N), _ptr(J, self.N), _ptr(x, 3 * self.N), _ptr(mu, 8 * self.N),
             _ptr(lam, 8 * self.N)]
        xd = _ptr(xdot, 3 * self.N)
        mem = _mem(*a, *([xd] if xdot is not None else []))
        self._check(lib().esmm_rhs_vjp(self.h, a[0][0], a[1][0], a[2][0], xd[0], a[3][0], a[4][0], mem))
        return lam

    def mesh_redistribute(self, dt=0.0):
        """(xdot, dtau, dt) as :meth:`Grid.mesh_redistribute`, in 3D."""
        xdot = np.empty(self._shape(3))
        tau, dtu = ctypes.c_double(), ctypes.c_double()
        self._check(lib().esmm_mesh_redistribute(self.h, float(dt), ctypes.c_void_p(xdot.ctypes.data),
                                                  ctypes.byref(tau), ctypes.byref(dtu), MEM_HOST))
        return xdot, tau.value, dtu.value


def _as_array(ptr, n):
    return None if not ptr else np.ctypeslib.as_array(ptr, shape=(int(n),))


class Slab(Grid):
    """One slab of a 2D grid decomposed along its second index
    (esmm_slab_create).  ``transport`` combines and exchanges host buffers
    between the slabs: an object with ``allreduce(buf, op)`` (in place, op
    OP_MAX / OP_MIN / OP_SUM) and ``exchange(send_lo, send_hi, recv_lo,
    recv_hi)`` (numpy arrays, None where the slab has no neighbour), e.g.
    :class:`paper_2107_12027_gb300.comm.LocalComm` or ``TorchComm``.  state_set
    takes the whole grid's arrays; state_get returns the slab's own rows."""

    def __init__(self, n, nslab, slab, transport, lo=(0.0, 0.0), hi=(1.0, 1.0), bc=(PERIODIC, PERIODIC),
                 gamma=5.0 / 3.0, p=2, w=5, stream=None, phys=RHD, scheme=None, **params):
        p, w = _apply_scheme(scheme, p, w, params)
        self.transport = transport

        def allreduce(ctx, buf, n_, op):
            try:
                transport.allreduce(_as_array(buf, n_), int(op))
                return 0
            except Exception:   # noqa: BLE001 -- reported to the library as a failed call
                return 1

        def exchange(ctx, slo, shi, rlo, rhi, count):
            try:
                transport.exchange(_as_array(slo, count), _as_array(shi, count), _as_array(rlo, count),
                                   _as_array(rhi, count))
                return 0
            except Exception:   # noqa: BLE001
                return 1
        self._fns = (ALLREDUCE_FN(allreduce), EXCHANGE_FN(exchange))   # kept alive with the handle
        self._comm = Comm(None, self._fns[0], self._fns[1])
        h = ctypes.c_void_p()
        nn = (ctypes.c_int * 2)(int(n[0]), int(n[1]))
        lo2 = (ctypes.c_double * 2)(lo[0], lo[1])
        hi2 = (ctypes.c_double * 2)(hi[0], hi[1])
        bc2 = (ctypes.c_int * 2)(bc[0], bc[1])
        st = ctypes.c_void_p(stream) if stream is not None else None
        self._check(lib().esmm_slab_create(ctypes.byref(h), nn, lo2, hi2, phys, bc2, int(nslab), int(slab),
                                           ctypes.byref(self._comm), st))
        self.h = h
        r = [ctypes.c_int() for _ in range(4)]
        self._check(lib().esmm_slab_rows(h, *[ctypes.byref(v) for v in r]))
        self.own0, self.own1, self.ext0, self.ext1 = (v.value for v in r)
        self.gnx, self.gny = int(n[0]), int(n[1])
        self.nx, self.ny = self.gnx, self.ext1 - self.ext0          # the held rows (esmm_rhs arrays)
        self.N = self.nx * self.ny
        self.phys = phys
        self.nv = 8 if phys == RMHD else 4
        self.set_eos(gamma)
        self.set_order(p, w)
        if params:
            self.set_params(**params)

    def state_set(self, prim, x=None):
        G = self.gnx * self.gny
        pp, mp = _ptr(prim, self.nv * G)
        px, mx = _ptr(x, 2 * G)
        self._check(lib().esmm_state_set(self.h, pp, px, _mem((pp, mp), (px, mx))))

    def state_get(self, what, out=None):
        size = {GET_PRIM: self.nv, GET_CONS: self.nv, GET_J: 1, GET_X: 2, GET_XDOT: 2}[what]
        rows = self.own1 - self.own0
        shape = (size, rows, self.nx) if size > 1 else (rows, self.nx)
        if out is None:
            out = np.empty(shape)
        po, mo = _ptr(out, size * rows * self.nx)
        self._check(lib().esmm_state_get(self.h, what, po, mo))
        return out


class Batch(Grid):
    """Many independent 2D RHD problems of different sizes in one handle.

    sizes: [(nx, ny), ...]; lo, hi, bc: one pair per problem or one shared."""

    def __init__(self, sizes, lo=(0.0, 0.0), hi=(1.0, 1.0), bc=(PERIODIC, PERIODIC), gamma=5.0 / 3.0, p=2, w=5,
                 stream=None, scheme=None, **params):
        p, w = _apply_scheme(scheme, p, w, params)
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        self.phys, self.nv = RHD, 4
        B = len(self.sizes)
        per = lambda v: [tuple(v)] * B if np.ndim(v) == 1 else [tuple(t) for t in v]
        los, his, bcs = per(lo), per(hi), per(bc)
        n = (ctypes.c_int * (2 * B))(*[k for s in self.sizes for k in s])
        lo2 = (ctypes.c_double * (2 * B))(*[k for s in los for k in s])
        hi2 = (ctypes.c_double * (2 * B))(*[k for s in his for k in s])
        bc2 = (ctypes.c_int * (2 * B))(*[int(k) for s in bcs for k in s])
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream is not None else None
        self._check(lib().esmm_batch_create(ctypes.byref(h), B, n, lo2, hi2, bc2, RHD, st))
        self.h = h
        self.nprob = B
        self.nx, self.ny, self.N = None, None, sum(a * b for a, b in self.sizes)
        self.set_eos(gamma)
        self.set_order(p, w)
        if params:
            self.set_params(**params)

    def state_set(self, b, prim, x=None):
        nx, ny = self.sizes[b]
        pp, mp = _ptr(prim, 4 * nx * ny)
        px, mx = _ptr(x, 2 * nx * ny)
        self._check(lib().esmm_batch_state_set(self.h, int(b), pp, px, _mem((pp, mp), (px, mx))))

    def state_get(self, b, what, out=None):
        nx, ny = self.sizes[b]
        size = {GET_PRIM: 4, GET_CONS: 4, GET_J: 1, GET_X: 2, GET_XDOT: 2}[what]
        if out is None:
            out = np.empty((size, ny, nx) if size > 1 else (ny, nx))
        po, mo = _ptr(out, size * nx * ny)
        self._check(lib().esmm_batch_state_get(self.h, int(b), what, po, mo))
        return out

    def times(self):
        t = (ctypes.c_double * self.nprob)()
        self._check(lib().esmm_batch_times(self.h, t))
        return np.array(t[:])

    def totals(self):
        out = (ctypes.c_double * (3 * self.nprob))()
        self._check(lib().esmm_batch_totals(self.h, out))
        return np.array(out[:]).reshape(self.nprob, 3)
