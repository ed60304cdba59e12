"""ctypes binding of librve (include/rve.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts NumPy arrays to the
C layout (Mandel component-major fields, float64) and back.  ``lib()`` loads the in-tree
``librve.so`` and raises if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librve.so")

RVE_OK = 0
RVE_E_ARG, RVE_E_OOM, RVE_E_NOCONV, RVE_E_CUDA, RVE_E_STATE, RVE_E_IO = -1, -2, -3, -4, -5, -6
RVE_SPLIT_SPECTRAL, RVE_SPLIT_NONE = 0, 1
RVE_GAMMA_ROTATED, RVE_GAMMA_CONTINUOUS = 0, 1
RVE_CONSTRAINT_LENGTH, RVE_CONSTRAINT_ENERGY = 0, 1
RVE_FP64, RVE_MIXED = 0, 1
RVE_FIELD_EPS, RVE_FIELD_EPS_T, RVE_FIELD_PHI, RVE_FIELD_H, RVE_FIELD_SIGMA = 0, 1, 2, 3, 4
RVE_CTRL_CRACK, RVE_CTRL_STRAIN = 0, 1

ERRORS = {RVE_E_ARG: "RVE_E_ARG", RVE_E_OOM: "RVE_E_OOM", RVE_E_NOCONV: "RVE_E_NOCONV",
          RVE_E_CUDA: "RVE_E_CUDA", RVE_E_STATE: "RVE_E_STATE", RVE_E_IO: "RVE_E_IO"}


class rve_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("n_phases", C.c_int),
                ("phase", C.POINTER(C.c_uint8)), ("E", C.POINTER(C.c_double)),
                ("nu", C.POINTER(C.c_double)), ("Gc", C.POINTER(C.c_double)),
                ("ell", C.c_double), ("f", C.c_double * 6), ("split", C.c_int),
                ("precision", C.c_int), ("k_res", C.c_double), ("alpha", C.c_double),
                ("newton_tol", C.c_double), ("krylov_tol", C.c_double),
                ("newton_max", C.c_int), ("krylov_max", C.c_int), ("gamma_op", C.c_int),
                ("constraint", C.c_int)]


class rve_step(C.Structure):
    _fields_ = [("E", C.c_double), ("sigma", C.c_double * 6), ("gamma", C.c_double),
                ("tau", C.c_double), ("newton_iters", C.c_int), ("krylov_iters", C.c_int),
                ("applies", C.c_int), ("err", C.c_double), ("cutbacks", C.c_int), ("fallbacks", C.c_int)]

    def as_dict(self):
        return dict(E=self.E, sigma=list(self.sigma), gamma=self.gamma, tau=self.tau,
                    newton_iters=self.newton_iters, krylov_iters=self.krylov_iters,
                    applies=self.applies, err=self.err, cutbacks=self.cutbacks, fallbacks=self.fallbacks)


class rve_result(C.Structure):
    _fields_ = [("id", C.c_longlong), ("status", C.c_int), ("n_increments", C.c_int),
                ("E", C.c_double), ("sigma", C.c_double * 6), ("gamma", C.c_double),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_end", C.c_double),
                ("footprint", C.c_longlong), ("error", C.c_char * 160)]

    def as_dict(self):
        return dict(id=self.id, status=self.status, n_increments=self.n_increments, E=self.E,
                    sigma=list(self.sigma), gamma=self.gamma, t_submit=self.t_submit,
                    t_start=self.t_start, t_end=self.t_end, footprint=self.footprint,
                    error=self.error.decode(errors="replace"))


_lib = None

# (name, restype, argtypes): every entry point of include/rve.h
SIGNATURES = [
    ("rve_desc_defaults", None, [C.POINTER(rve_desc)]),
    ("rve_create", C.c_int, [C.POINTER(rve_desc), C.POINTER(C.c_void_p)]),
    ("rve_set_notch", C.c_int, [C.c_void_p, C.POINTER(C.c_uint8)]),
    ("rve_startup", C.c_int, [C.c_void_p, C.c_double, C.POINTER(rve_step)]),
    ("rve_crack_increment", C.c_int, [C.c_void_p, C.c_double, C.POINTER(rve_step)]),
    ("rve_strain_increment", C.c_int, [C.c_void_p, C.c_double, C.POINTER(rve_step)]),
    ("rve_staggered_increment", C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.POINTER(rve_step),
                                          C.POINTER(C.c_int)]),
    ("rve_get_macro_stress", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("rve_get_fields", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_size_t]),
    ("rve_set_state", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.c_double, C.c_double]),
    ("rve_autotune", C.c_int, [C.c_void_p]),
    ("rve_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("rve_info", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                           C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    ("rve_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("rve_load", C.c_int, [C.c_char_p, C.POINTER(C.c_void_p)]),
    ("rve_destroy", None, [C.c_void_p]),
    ("rve_last_error", C.c_char_p, [C.c_void_p]),
    ("rve_linearize", C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    ("rve_residual", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(C.c_double)]),
    ("rve_apply", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double,
                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("rve_apply_device", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rve_apply_device_batch", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p),
                                         C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    ("rve_apply_device_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("rve_kernel_launches", C.c_longlong, [C.c_void_p]),
    ("rve_batch_crack_increment", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_double),
                                            C.POINTER(rve_step), C.POINTER(C.c_int)]),
    ("rve_footprint", C.c_int, [C.POINTER(rve_desc), C.POINTER(C.c_longlong)]),
    ("rve_effective_toughness", C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.c_double,
                                          C.c_double, C.POINTER(C.c_double)]),
    ("rve_j_integral", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    ("rve_server_create", C.c_int, [C.c_longlong, C.c_int, C.POINTER(C.c_void_p)]),
    ("rve_server_submit", C.c_int, [C.c_void_p, C.POINTER(rve_desc), C.POINTER(C.c_uint8), C.c_int,
                                    C.c_double, C.POINTER(C.c_longlong)]),
    ("rve_server_poll", C.c_int, [C.c_void_p, C.POINTER(rve_result), C.c_int, C.POINTER(C.c_int)]),
    ("rve_server_drain", C.c_int, [C.c_void_p]),
    ("rve_server_stats", C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                   C.POINTER(C.c_int)]),
    ("rve_server_destroy", None, [C.c_void_p]),
]


def lib():
    """Load librve.so (in-tree build).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2412_17445_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class RVEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def mandel_from_tensor(t: np.ndarray) -> np.ndarray:
    """(shape + (d, d)) symmetric tensors -> (m, n) Mandel component-major."""
    d = t.shape[-1]
    f = t.reshape(-1, d, d)
    r2 = np.sqrt(2.0)
    if d == 2:
        comps = [f[:, 0, 0], f[:, 1, 1], r2 * f[:, 0, 1]]
    else:
        comps = [f[:, 0, 0], f[:, 1, 1], f[:, 2, 2], r2 * f[:, 1, 2], r2 * f[:, 0, 2], r2 * f[:, 0, 1]]
    return np.ascontiguousarray(np.stack(comps))


def tensor_from_mandel(mv: np.ndarray, shape) -> np.ndarray:
    """(m, n) Mandel -> shape + (d, d) symmetric tensors."""
    m = mv.shape[0]
    d = 2 if m == 3 else 3
    t = np.zeros((mv.shape[1], d, d))
    h = 1.0 / np.sqrt(2.0)
    if d == 2:
        t[:, 0, 0], t[:, 1, 1] = mv[0], mv[1]
        t[:, 0, 1] = t[:, 1, 0] = h * mv[2]
    else:
        t[:, 0, 0], t[:, 1, 1], t[:, 2, 2] = mv[0], mv[1], mv[2]
        t[:, 1, 2] = t[:, 2, 1] = h * mv[3]
        t[:, 0, 2] = t[:, 2, 0] = h * mv[4]
        t[:, 0, 1] = t[:, 1, 0] = h * mv[5]
    return t.reshape(tuple(shape) + (d, d))


def mandel_vector(f: np.ndarray) -> np.ndarray:
    """d x d tensor -> Mandel 6-vector (unused entries 0)."""
    out = np.zeros(6)
    mv = mandel_from_tensor(np.asarray(f, float)[None])
    out[: mv.shape[0]] = mv[:, 0]
    return out


def make_desc(inp, precision=RVE_FP64, split=RVE_SPLIT_SPECTRAL, newton_tol=1e-10, krylov_tol=None,
              newton_max=50, krylov_max=4000, alpha=1.0, k_res=0.0, gamma_op=0, constraint=0):
    """rve_desc for an RVE input; returns (desc, keep) where keep holds the arrays the
    descriptor points to (keep it alive while the descriptor is used)."""
    d = rve_desc()
    lib().rve_desc_defaults(C.byref(d))
    shp = tuple(inp.shape)
    if len(shp) == 2:
        d.nz, d.ny, d.nx = 1, shp[0], shp[1]
    else:
        d.nz, d.ny, d.nx = shp
    keep = dict(phase=np.ascontiguousarray(inp.phase, dtype=np.uint8).reshape(-1),
                E=np.ascontiguousarray(inp.E, dtype=np.float64),
                nu=np.ascontiguousarray(inp.nu, dtype=np.float64),
                Gc=np.ascontiguousarray(inp.Gc, dtype=np.float64),
                notch=np.ascontiguousarray(inp.notch, dtype=np.uint8).reshape(-1))
    d.n_phases = len(keep["E"])
    d.phase = keep["phase"].ctypes.data_as(C.POINTER(C.c_uint8))
    d.E, d.nu, d.Gc = _dp(keep["E"]), _dp(keep["nu"]), _dp(keep["Gc"])
    d.ell = float(inp.ell)
    fm = mandel_vector(inp.f)
    for k in range(6):
        d.f[k] = fm[k]
    d.split, d.precision, d.k_res, d.alpha = split, precision, k_res, alpha
    d.newton_tol = newton_tol
    d.krylov_tol = krylov_tol if krylov_tol is not None else (1e-10 if precision == RVE_FP64 else 1e-2)
    d.newton_max, d.krylov_max = newton_max, krylov_max
    d.gamma_op = gamma_op
    d.constraint = constraint
    return d, keep


def apply_device_batch(rves, xs, xEs, ys, yEs):
    """rve_apply_device_batch: scaled applies of several RVEs of one shape in single launches
    (device pointers, e.g. torch tensors' data_ptr())."""
    n = len(rves)
    arr = lambda v: (C.c_void_p * n)(*[C.c_void_p(p) for p in v])
    hs = (C.c_void_p * n)(*[g.h.value if isinstance(g.h, C.c_void_p) else g.h for g in rves])
    rc = lib().rve_apply_device_batch(hs, n, arr(xs), arr(xEs), arr(ys), arr(yEs))
    if rc != RVE_OK:
        raise RVEError(rc, "rve_apply_device_batch")


def effective_toughness(E, sigma_f, area: float, length: float) -> float:
    """rve_effective_toughness (Eq. JaviGc) on host arrays."""
    e = np.ascontiguousarray(E, dtype=np.float64)
    s = np.ascontiguousarray(sigma_f, dtype=np.float64)
    G = C.c_double()
    rc = lib().rve_effective_toughness(_dp(e), _dp(s), len(e), float(area), float(length), C.byref(G))
    if rc != RVE_OK:
        raise RVEError(rc, "rve_effective_toughness")
    return G.value


def footprint(inp, precision=RVE_FP64, constraint=RVE_CONSTRAINT_LENGTH) -> int:
    d, keep = make_desc(inp, precision, constraint=constraint)
    b = C.c_longlong()
    rc = lib().rve_footprint(C.byref(d), C.byref(b))
    if rc != RVE_OK:
        raise RVEError(rc, "rve_footprint")
    return b.value


class Server:
    """Continuous-batching server (rve_server_*): submit requests, drain, poll results."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 64):
        h = C.c_void_p()
        rc = lib().rve_server_create(int(hbm_budget_bytes), int(max_active), C.byref(h))
        if rc != RVE_OK:
            raise RVEError(rc, "rve_server_create")
        self.h = h

    def submit(self, inp, n_increments: int, da: float = 1.0, **kw) -> int:
        d, keep = make_desc(inp, **kw)
        rid = C.c_longlong()
        notch = keep["notch"].ctypes.data_as(C.POINTER(C.c_uint8)) if np.any(keep["notch"]) else None
        rc = lib().rve_server_submit(self.h, C.byref(d), notch, int(n_increments), float(da), C.byref(rid))
        if rc != RVE_OK:
            raise RVEError(rc, "rve_server_submit")
        return rid.value

    def drain(self):
        lib().rve_server_drain(self.h)

    def poll(self, max_results: int = 1024):
        buf = (rve_result * max_results)()
        n = C.c_int()
        lib().rve_server_poll(self.h, buf, max_results, C.byref(n))
        return [buf[i].as_dict() for i in range(n.value)]

    def stats(self):
        used, act, q = C.c_longlong(), C.c_int(), C.c_int()
        lib().rve_server_stats(self.h, C.byref(used), C.byref(act), C.byref(q))
        return dict(hbm_in_use=used.value, active=act.value, queued=q.value)

    def close(self):
        if getattr(self, "h", None):
            lib().rve_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RVE:
    """One RVE on the GPU (a handle of librve)."""

    def __init__(self, inp, precision: int = RVE_FP64, split: int = RVE_SPLIT_SPECTRAL,
                 newton_tol: float = 1e-10, krylov_tol: Optional[float] = None,
                 newton_max: int = 50, krylov_max: int = 4000, alpha: float = 1.0,
                 k_res: float = 0.0, notch: bool = True, handle=None, gamma_op: int = RVE_GAMMA_ROTATED,
                 constraint: int = RVE_CONSTRAINT_LENGTH):
        L = lib()
        self.shape = tuple(inp.shape) if inp is not None else None
        if handle is not None:
            self.h = handle
        else:
            d = rve_desc()
            L.rve_desc_defaults(C.byref(d))
            shp = tuple(inp.shape)
            if len(shp) == 2:
                d.nz, d.ny, d.nx = 1, shp[0], shp[1]
            else:
                d.nz, d.ny, d.nx = shp
            self._phase = np.ascontiguousarray(inp.phase, dtype=np.uint8).reshape(-1)
            self._E = np.ascontiguousarray(inp.E, dtype=np.float64)
            self._nu = np.ascontiguousarray(inp.nu, dtype=np.float64)
            self._Gc = np.ascontiguousarray(inp.Gc, dtype=np.float64)
            d.n_phases = len(self._E)
            d.phase = self._phase.ctypes.data_as(C.POINTER(C.c_uint8))
            d.E, d.nu, d.Gc = _dp(self._E), _dp(self._nu), _dp(self._Gc)
            d.ell = float(inp.ell)
            fm = mandel_vector(inp.f)
            for k in range(6):
                d.f[k] = fm[k]
            d.split = split
            d.precision = precision
            d.k_res = k_res
            d.alpha = alpha
            d.newton_tol = newton_tol
            d.krylov_tol = krylov_tol if krylov_tol is not None else (1e-10 if precision == RVE_FP64 else 1e-2)
            d.newton_max = newton_max
            d.krylov_max = krylov_max
            d.gamma_op = gamma_op
            d.constraint = constraint
            h = C.c_void_p()
            self._check(L.rve_create(C.byref(d), C.byref(h)), None)
            self.h = h
            if notch and inp.notch is not None and np.any(inp.notch):
                m = np.ascontiguousarray(inp.notch, dtype=np.uint8).reshape(-1)
                self._check(L.rve_set_notch(self.h, m.ctypes.data_as(C.POINTER(C.c_uint8))))
        dim, m, n, prec = C.c_int(), C.c_int(), C.c_longlong(), C.c_int()
        L.rve_info(self.h, C.byref(dim), C.byref(m), C.byref(n), C.byref(prec))
        self.dim, self.m, self.n, self.precision = dim.value, m.value, n.value, prec.value

    # -- helpers ------------------------------------------------------------------------
    def _check(self, rc, h="self"):
        if rc != RVE_OK:
            L = lib()
            msg = L.rve_last_error(self.h if h == "self" else None)
            raise RVEError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            lib().rve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- solver ---------------------------------------------------------------------------
    def set_stream(self, stream_ptr: int):
        self._check(lib().rve_set_stream(self.h, C.c_void_p(stream_ptr)))

    def startup(self, beta: float = 0.25):
        st = rve_step()
        self._check(lib().rve_startup(self.h, beta, C.byref(st)))
        return st.as_dict()

    def staggered_increment(self, E_target: float, tol: float = 1e-10, max_sweeps: int = 200):
        """rve_staggered_increment (Algorithm 1); the step record gains "sweeps"."""
        st = rve_step()
        sw = C.c_int()
        self._check(lib().rve_staggered_increment(self.h, float(E_target), float(tol), int(max_sweeps),
                                                  C.byref(st), C.byref(sw)))
        d = st.as_dict()
        d["sweeps"] = sw.value
        return d

    def crack_increment(self, da: float):
        st = rve_step()
        self._check(lib().rve_crack_increment(self.h, float(da), C.byref(st)))
        return st.as_dict()

    def strain_increment(self, E: float):
        st = rve_step()
        self._check(lib().rve_strain_increment(self.h, float(E), C.byref(st)))
        return st.as_dict()

    def macro_stress(self):
        s = np.zeros(6)
        E = C.c_double()
        self._check(lib().rve_get_macro_stress(self.h, _dp(s), C.byref(E)))
        return s[: self.m].copy(), E.value

    def field(self, which: int) -> np.ndarray:
        cnt = self.n * (self.m if which in (RVE_FIELD_EPS, RVE_FIELD_EPS_T, RVE_FIELD_SIGMA) else 1)
        out = np.zeros(cnt)
        self._check(lib().rve_get_fields(self.h, which, _dp(out), cnt))
        if cnt > self.n:
            return out.reshape(self.m, self.n)
        return out

    def j_integral(self, box) -> float:
        """rve_j_integral: J of the committed state around the rectangle of voxel centres
        box = (x0, y0, x1, y1) (2D)."""
        x0, y0, x1, y1 = (int(v) for v in box)
        J = C.c_double()
        self._check(lib().rve_j_integral(self.h, x0, y0, x1, y1, C.byref(J)))
        return J.value

    def set_state(self, eps_t_mandel: np.ndarray, phi: np.ndarray, H: np.ndarray, E: float, tau: float = 0.0):
        e = np.ascontiguousarray(eps_t_mandel, dtype=np.float64).reshape(-1)
        p = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        hh = np.ascontiguousarray(H, dtype=np.float64).reshape(-1)
        self._check(lib().rve_set_state(self.h, _dp(e), _dp(p), _dp(hh), float(E), float(tau)))

    def linearize(self, control: int, target: float):
        self._check(lib().rve_linearize(self.h, control, float(target)))

    def residual(self):
        F1 = np.zeros(self.m * self.n)
        F2 = np.zeros(self.n)
        F3 = C.c_double()
        self._check(lib().rve_residual(self.h, _dp(F1), _dp(F2), C.byref(F3)))
        return F1.reshape(self.m, self.n), F2, F3.value

    def apply(self, d_eps_mandel: np.ndarray, d_phi: np.ndarray, dE: float):
        de = np.ascontiguousarray(d_eps_mandel, dtype=np.float64).reshape(-1)
        dp = np.ascontiguousarray(d_phi, dtype=np.float64).reshape(-1)
        oe = np.zeros(self.m * self.n)
        op = np.zeros(self.n)
        oE = C.c_double()
        self._check(lib().rve_apply(self.h, _dp(de), _dp(dp), float(dE), _dp(oe), _dp(op), C.byref(oE)))
        return oe.reshape(self.m, self.n), op, oE.value

    def apply_device(self, x_ptr: int, xE_ptr: int, y_ptr: int, yE_ptr: int):
        """Scaled apply on device buffers (e.g. torch tensors' data_ptr())."""
        self._check(lib().rve_apply_device(self.h, C.c_void_p(x_ptr), C.c_void_p(xE_ptr),
                                           C.c_void_p(y_ptr), C.c_void_p(yE_ptr)))

    def autotune(self):
        self._check(lib().rve_autotune(self.h))

    def kernel_launches(self) -> int:
        return int(lib().rve_kernel_launches(self.h))

    def save(self, path: str):
        self._check(lib().rve_save(self.h, path.encode()))

    @classmethod
    def load(cls, path: str, shape=None):
        h = C.c_void_p()
        rc = lib().rve_load(path.encode(), C.byref(h))
        if rc != RVE_OK:
            raise RVEError(rc, lib().rve_last_error(None).decode())
        obj = cls.__new__(cls)
        RVE.__init__(obj, None, handle=h)
        obj.shape = shape
        return obj


def batch_crack_increment(rves, da):
    """rve_batch_crack_increment over several handles; returns (results, statuses)."""
    n = len(rves)
    hs = (C.c_void_p * n)(*[r.h for r in rves])
    das = (C.c_double * n)(*[float(x) for x in da])
    out = (rve_step * n)()
    st = (C.c_int * n)()
    lib().rve_batch_crack_increment(hs, n, das, out, st)
    return [o.as_dict() for o in out], list(st)
