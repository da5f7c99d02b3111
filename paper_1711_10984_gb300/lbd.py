"""ctypes binding of ``liblbd.so`` (C ABI in ``include/lbd.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  ``load()`` raises if the library has not been built (there is no CPU
fallback).  ``Sim`` wraps one context; the module-level functions keep the C
names for callers that want the raw ABI.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbd.so")

LBD_OK, LBD_EINVAL, LBD_ENOMEM, LBD_ECUDA = 0, -1, -2, -3
LBD_ENONFINITE, LBD_EUNSTABLE, LBD_ETIMEOUT = -4, -5, -6
LBD_FP64, LBD_FP32 = 0, 1
LBD_FROZEN_U, LBD_BODY_FORCE, LBD_WALLS = 1, 2, 16
LBD_MAX_SOURCES = 64

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


class lbd_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32)]


class lbd_source(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("R", ctypes.c_double)]


class lbd_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("b", ctypes.c_double), ("B0", ctypes.c_double),
                ("B1", ctypes.c_double), ("M", ctypes.c_double), ("D", ctypes.c_double),
                ("tau", ctypes.c_double), ("gamma", ctypes.c_double), ("c0", ctypes.c_double),
                ("A0", ctypes.c_double), ("A_max", ctypes.c_double), ("t_on", ctypes.c_int64),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("ux0", ctypes.c_double),
                ("uy0", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("precision", ctypes.c_int32), ("n_src", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("src", lbd_source * LBD_MAX_SOURCES)]


class lbd_diag(ctypes.Structure):
    _fields_ = [("sum_rho", ctypes.c_double), ("sum_phi", ctypes.c_double),
                ("sum_psi", ctypes.c_double), ("cm_x", ctypes.c_double),
                ("cm_y", ctypes.c_double), ("mass_pos", ctypes.c_double),
                ("min_B", ctypes.c_double), ("min_psi", ctypes.c_double),
                ("nonfinite", ctypes.c_int64)]


class lbd_droplet(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("mass", ctypes.c_double),
                ("ux", ctypes.c_double), ("uy", ctypes.c_double), ("sites", ctypes.c_int64)]


LBD_MAX_DROPLETS = 64


class lbd_droplet_init(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("x", "y", "R", "psi_mean", "psi_noise", "gx", "gy")]

_P = ctypes.c_void_p
# name -> (restype, argtypes); the list mirrors include/lbd.h
SIGNATURES = {
    "lbd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbd_last_error": (ctypes.c_char_p, [_P]),
    "lbd_create": (ctypes.c_int, [ctypes.POINTER(lbd_grid), ctypes.POINTER(lbd_params), _P,
                                  ctypes.POINTER(_P)]),
    "lbd_set_params": (ctypes.c_int, [_P, ctypes.POINTER(lbd_params)]),
    "lbd_set_fields": (ctypes.c_int, [_P, _dp, _dp, _dp, _dp, _dp]),
    "lbd_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbd_get_fields": (ctypes.c_int, [_P, _dp, _dp, _dp, _dp, _dp]),
    "lbd_set_fields_f32": (ctypes.c_int, [_P, _fp, _fp, _fp, _fp, _fp]),
    "lbd_get_fields_f32": (ctypes.c_int, [_P, _fp, _fp, _fp, _fp, _fp]),
    "lbd_get_populations": (ctypes.c_int, [_P, _dp]),
    "lbd_diagnostics": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(lbd_diag)]),
    "lbd_droplets": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(lbd_droplet)]),
    "lbd_squirmer": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(lbd_droplet),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int64)]),
    "lbd_get_fields_device": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "lbd_set_populations": (ctypes.c_int, [_P, _dp]),
    "lbd_init_droplets": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(lbd_droplet_init),
                                         ctypes.c_double, ctypes.c_double, ctypes.c_uint64]),
    "lbd_set_tile": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "lbd_tiles": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.c_int32]),
    "lbd_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)]),
    "lbd_diagnostics_static": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                              ctypes.c_int32, _P, _P, _P, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              _P, ctypes.POINTER(lbd_diag)]),
    "lbd_adjoint": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                   _dp, _dp, _dp]),
    "lbd_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(lbd_grid),
                                        ctypes.POINTER(lbd_params), _P, ctypes.POINTER(_P)]),
    "lbd_batch_last_error": (ctypes.c_char_p, [_P]),
    "lbd_batch_set_fields": (ctypes.c_int, [_P, ctypes.c_int32, _dp, _dp, _dp, _dp, _dp]),
    "lbd_batch_get_fields": (ctypes.c_int, [_P, ctypes.c_int32, _dp, _dp, _dp, _dp, _dp]),
    "lbd_batch_diagnostics": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                             ctypes.POINTER(lbd_diag)]),
    "lbd_batch_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbd_batch_set_tile": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "lbd_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "lbd_batch_synchronize": (ctypes.c_int, [_P]),
    "lbd_batch_get_tile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "lbd_get_tile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)]),
    "lbd_batch_get_time": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "lbd_batch_destroy": (None, [_P]),
    "lbd_get_time": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "lbd_set_time": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbd_synchronize": (ctypes.c_int, [_P]),
    "lbd_set_check": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbd_debug_fail_alloc": (ctypes.c_int, [ctypes.c_int32]),
    "lbd_fp64_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "lbd_destroy": (None, [_P]),
}

_lib = None


class LbdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (lib().lbd_strerror(code).decode(), msg))
        self.code = code


def load(path=LIB_PATH):
    """Load the CUDA library; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("liblbd.so is not built; run __graft_entry__.build() or "
                               "python paper_1711_10984_gb300/build.py")
        l = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(l, name)
            fn.restype = res
            fn.argtypes = args
        _lib = l
    return _lib


lib = load


def _arr(a, n):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a, a.ctypes.data_as(_dp)


def make_params(precision=LBD_FP64, sources=(), flags=0, **kw):
    p = lbd_params()
    defaults = dict(a=-0.001, b=0.001, B0=0.006, B1=-0.05, M=1.0, D=0.1, tau=1.0, gamma=0.0,
                    c0=0.0, A0=0.0, A_max=0.0, t_on=0, fx=0.0, fy=0.0, ux0=0.0, uy0=0.0)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(p, k, int(v) if k == "t_on" else float(v))
    p.flags = int(flags)
    p.precision = int(precision)
    sources = list(sources)
    if len(sources) > LBD_MAX_SOURCES:
        raise ValueError("at most %d sources" % LBD_MAX_SOURCES)
    p.n_src = len(sources)
    for k, (x, y, R) in enumerate(sources):
        p.src[k] = lbd_source(float(x), float(y), float(R))
    return p


def tiles():
    """Tile shapes (bx, by) compiled into the library."""
    bx = (ctypes.c_int32 * 64)()
    by = (ctypes.c_int32 * 64)()
    n = load().lbd_tiles(bx, by, 64)
    return [(bx[k], by[k]) for k in range(n)]


class Sim:
    """One solver context on the current CUDA device."""

    def __init__(self, nx, ny, precision=LBD_FP64, sources=(), flags=0, stream=None, **kw):
        self.nx, self.ny = int(nx), int(ny)
        self.N = self.nx * self.ny
        self.params = make_params(precision, sources, flags, **kw)
        self._h = _P()
        g = lbd_grid(self.nx, self.ny)
        rc = load().lbd_create(ctypes.byref(g), ctypes.byref(self.params),
                               ctypes.c_void_p(stream or 0), ctypes.byref(self._h))
        if rc != LBD_OK:
            raise LbdError(rc, "lbd_create failed")

    def _check(self, rc):
        if rc != LBD_OK:
            raise LbdError(rc, load().lbd_last_error(self._h).decode())

    def set_params(self, precision=None, sources=(), flags=0, **kw):
        prec = self.params.precision if precision is None else precision
        self.params = make_params(prec, sources, flags, **kw)
        self._check(load().lbd_set_params(self._h, ctypes.byref(self.params)))

    def set_fields(self, phi, psi, rho=None, ux=None, uy=None):
        arrs = [_arr(a, self.N) for a in (rho, ux, uy, phi, psi)]
        self._check(load().lbd_set_fields(self._h, *[p for _, p in arrs]))

    def step(self, n=1):
        self._check(load().lbd_step(self._h, int(n)))
        return self

    def set_fields_f32(self, phi, psi, rho=None, ux=None, uy=None):
        """lbd_set_fields_f32: the fields as float32 host arrays."""
        def arr(a):
            if a is None:
                return None, None
            a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
            if a.size != self.N:
                raise ValueError("expected %d values" % self.N)
            return a, a.ctypes.data_as(_fp)
        arrs = [arr(a) for a in (rho, ux, uy, phi, psi)]
        self._check(load().lbd_set_fields_f32(self._h, *[q for _, q in arrs]))

    def fields_f32(self):
        """lbd_get_fields_f32: (rho, ux, uy, phi, psi) as (ny, nx) float32 arrays."""
        out = [np.empty(self.N, dtype=np.float32) for _ in range(5)]
        self._check(load().lbd_get_fields_f32(self._h, *[o.ctypes.data_as(_fp) for o in out]))
        return tuple(o.reshape(self.ny, self.nx) for o in out)

    def fields(self):
        """(rho, ux, uy, phi, psi) as (ny, nx) float64 arrays."""
        out = [np.empty(self.N) for _ in range(5)]
        self._check(load().lbd_get_fields(self._h, *[o.ctypes.data_as(_dp) for o in out]))
        return tuple(o.reshape(self.ny, self.nx) for o in out)

    def init_droplets(self, droplets, psi_bg=0.1, xi=0.0, seed=0):
        """lbd_init_droplets: droplets as dicts with keys x, y, R and optional
        psi_mean (default psi_bg), noise, gx, gy (the recipe of
        inputs.droplet_fields)."""
        n = len(droplets)
        arr = (lbd_droplet_init * n)(*[lbd_droplet_init(
            d["x"], d["y"], d["R"], d.get("psi_mean", psi_bg), d.get("noise", 0.0),
            d.get("gx", 0.0), d.get("gy", 0.0)) for d in droplets])
        self._check(load().lbd_init_droplets(self._h, n, arr, float(psi_bg), float(xi),
                                             int(seed) & 0xFFFFFFFFFFFFFFFF))

    def fields_device(self, rho=0, ux=0, uy=0, phi=0, psi=0):
        """lbd_get_fields_device into caller-owned device buffers given as raw
        addresses (0 = skip), e.g. torch tensors' data_ptr()."""
        ptrs = [ctypes.c_void_p(int(a)) if a else None for a in (rho, ux, uy, phi, psi)]
        self._check(load().lbd_get_fields_device(self._h, *ptrs))

    def set_populations(self, f):
        """lbd_set_populations from an array shaped like populations()."""
        a = np.ascontiguousarray(f, dtype=np.float64).ravel()
        if a.size != 9 * self.N:
            raise ValueError("expected %d values" % (9 * self.N))
        self._check(load().lbd_set_populations(self._h, a.ctypes.data_as(_dp)))

    def populations(self):
        f = np.empty(9 * self.N)
        self._check(load().lbd_get_populations(self._h, f.ctypes.data_as(_dp)))
        return f.reshape(9, self.ny, self.nx)

    def diagnostics(self, refx, refy, check=False):
        """lbd_diagnostics as a dict; its verdict (LBD_OK, LBD_ENONFINITE or
        LBD_EUNSTABLE) is under "status", and check=True raises on a bad one."""
        d = lbd_diag()
        rc = load().lbd_diagnostics(self._h, float(refx), float(refy), ctypes.byref(d))
        if rc not in (LBD_OK, LBD_ENONFINITE, LBD_EUNSTABLE) or (check and rc != LBD_OK):
            self._check(rc)
        out = {k: getattr(d, k) for k, _ in lbd_diag._fields_}
        out["status"] = rc
        return out

    def set_check(self, every):
        """lbd_set_check: run-time checks every `every` steps (0 = off)."""
        self._check(load().lbd_set_check(self._h, int(every)))

    def droplets(self, refs):
        """Per-droplet centre, mass, mean velocity and site count (lbd_droplets)
        for the reference points refs = [(x, y), ...]."""
        n = len(refs)
        ref = (ctypes.c_double * (2 * n))(*[float(v) for r in refs for v in r])
        out = (lbd_droplet * n)()
        self._check(load().lbd_droplets(self._h, n, ref, out))
        return [{k: getattr(d, k) for k, _ in lbd_droplet._fields_} for d in out]

    def squirmer(self, drops):
        """Squirmer fit of Eq. (21) (lbd_squirmer) for droplets as returned by
        droplets(): list of dict(b1, b2, points)."""
        n = len(drops)
        arr = (lbd_droplet * n)(*[lbd_droplet(d["x"], d["y"], d.get("mass", 0.0), d["ux"],
                                              d["uy"], int(d.get("sites", 0))) for d in drops])
        b1, b2 = (ctypes.c_double * n)(), (ctypes.c_double * n)()
        pts = (ctypes.c_int64 * n)()
        self._check(load().lbd_squirmer(self._h, n, arr, b1, b2, pts))
        return [dict(b1=b1[k], b2=b2[k], points=pts[k]) for k in range(n)]

    @property
    def t(self):
        v = ctypes.c_int64()
        self._check(load().lbd_get_time(self._h, ctypes.byref(v)))
        return v.value

    @t.setter
    def t(self, value):
        self._check(load().lbd_set_time(self._h, int(value)))

    def set_tile(self, bx, by):
        self._check(load().lbd_set_tile(self._h, int(bx), int(by)))

    def autotune(self, reps=20):
        """Time every compiled tile on the current state; keep and return the fastest."""
        bx, by = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().lbd_autotune(self._h, int(reps), ctypes.byref(bx), ctypes.byref(by)))
        return bx.value, by.value

    def adjoint(self, nsteps, ckpt_every, refx, want_dpsi=True):
        """Run nsteps from the current state; return (L, dL/dpsi0 or None, dL/dB1)
        for L = X_cm(end) - X_cm(start) (see lbd_adjoint)."""
        loss, dB1 = ctypes.c_double(), ctypes.c_double()
        dpsi = np.empty(self.N) if want_dpsi else None
        self._check(load().lbd_adjoint(self._h, int(nsteps), int(ckpt_every), float(refx),
                                       ctypes.byref(loss),
                                       dpsi.ctypes.data_as(_dp) if want_dpsi else None,
                                       ctypes.byref(dB1)))
        return loss.value, (dpsi.reshape(self.ny, self.nx) if want_dpsi else None), dB1.value

    def synchronize(self):
        self._check(load().lbd_synchronize(self._h))

    @property
    def tile(self):
        """The current launch shape (bx, by)."""
        bx, by = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().lbd_get_tile(self._h, ctypes.byref(bx), ctypes.byref(by)))
        return bx.value, by.value

    def close(self):
        if self._h:
            load().lbd_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent instances (own lattice and parameters each) stepped together
    by one persistent launch per step, replayed from CUDA graphs."""

    def __init__(self, grids, params, stream=None):
        self.n = len(grids)
        self.grids = [(int(nx), int(ny)) for nx, ny in grids]
        g = (lbd_grid * self.n)(*[lbd_grid(nx, ny) for nx, ny in self.grids])
        p = (lbd_params * self.n)(*params)
        self._h = _P()
        rc = load().lbd_batch_create(self.n, g, p, ctypes.c_void_p(stream or 0),
                                     ctypes.byref(self._h))
        if rc != LBD_OK:
            raise LbdError(rc, "lbd_batch_create failed")

    def _check(self, rc):
        if rc != LBD_OK:
            raise LbdError(rc, load().lbd_batch_last_error(self._h).decode())

    def set_fields(self, k, phi, psi, rho=None, ux=None, uy=None):
        N = self.grids[k][0] * self.grids[k][1]
        arrs = [_arr(a, N) for a in (rho, ux, uy, phi, psi)]
        self._check(load().lbd_batch_set_fields(self._h, int(k), *[q for _, q in arrs]))

    def fields(self, k):
        nx, ny = self.grids[k]
        out = [np.empty(nx * ny) for _ in range(5)]
        self._check(load().lbd_batch_get_fields(self._h, int(k), *[o.ctypes.data_as(_dp) for o in out]))
        return tuple(o.reshape(ny, nx) for o in out)

    def diagnostics(self, k, refx, refy):
        d = lbd_diag()
        rc = load().lbd_batch_diagnostics(self._h, int(k), float(refx), float(refy),
                                          ctypes.byref(d))
        if rc not in (LBD_OK, LBD_ENONFINITE, LBD_EUNSTABLE):
            self._check(rc)
        out = {kk: getattr(d, kk) for kk, _ in lbd_diag._fields_}
        out["status"] = rc
        return out

    def step(self, n=1):
        self._check(load().lbd_batch_step(self._h, int(n)))
        return self

    def set_tile(self, bx, by):
        self._check(load().lbd_batch_set_tile(self._h, int(bx), int(by)))

    def autotune(self, reps=5):
        bx, by = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().lbd_batch_autotune(self._h, int(reps), ctypes.byref(bx), ctypes.byref(by)))
        return bx.value, by.value

    def synchronize(self):
        self._check(load().lbd_batch_synchronize(self._h))

    @property
    def tile(self):
        """The current launch shape (bx, by)."""
        bx, by = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().lbd_batch_get_tile(self._h, ctypes.byref(bx), ctypes.byref(by)))
        return bx.value, by.value

    @property
    def t(self):
        v = ctypes.c_int64()
        self._check(load().lbd_batch_get_time(self._h, ctypes.byref(v)))
        return v.value

    def close(self):
        if self._h:
            load().lbd_batch_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
