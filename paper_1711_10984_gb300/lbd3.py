"""ctypes binding of the 3D coupled step (include/lbd3.h): argument marshalling
only, every step runs in the CUDA library.  Arrays are (nz, ny, nx) float64."""
import ctypes

import numpy as np

from . import lbd

_dp = ctypes.POINTER(ctypes.c_double)
_P = ctypes.c_void_p


class lbd3_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class lbd3_source(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("z", ctypes.c_double),
                ("R", ctypes.c_double)]


class lbd3_params(ctypes.Structure):
    _fields_ = [("base", lbd.lbd_params), ("fz", ctypes.c_double), ("uz0", ctypes.c_double),
                ("n_src", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("src", lbd3_source * lbd.LBD_MAX_SOURCES)]


class lbd3_diag(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("sum_rho", "sum_phi", "sum_psi", "cm_x", "cm_y",
                                               "cm_z", "mass_pos")] + [("nonfinite", ctypes.c_int64)]


SIGNATURES = {
    "lbd3_create": (ctypes.c_int, [ctypes.POINTER(lbd3_grid), ctypes.POINTER(lbd3_params), _P,
                                   ctypes.POINTER(_P)]),
    "lbd3_last_error": (ctypes.c_char_p, [_P]),
    "lbd3_set_params": (ctypes.c_int, [_P, ctypes.POINTER(lbd3_params)]),
    "lbd3_set_fields": (ctypes.c_int, [_P] + [_dp] * 6),
    "lbd3_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbd3_get_fields": (ctypes.c_int, [_P] + [_dp] * 6),
    "lbd3_get_populations": (ctypes.c_int, [_P, _dp]),
    "lbd3_diagnostics": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.POINTER(lbd3_diag)]),
    "lbd3_synchronize": (ctypes.c_int, [_P]),
    "lbd3_get_time": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "lbd3_set_zrun": (ctypes.c_int, [_P, ctypes.c_int32]),
    "lbd3_get_zrun": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "lbd3_destroy": (None, [_P]),
}

_ready = False


def load():
    global _ready
    lib = lbd.load()
    if not _ready:
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _ready = True
    return lib


def make_params(precision=lbd.LBD_FP64, sources=(), flags=0, fz=0.0, uz0=0.0, **kw):
    p = lbd3_params()
    p.base = lbd.make_params(precision, (), flags, **kw)
    p.fz, p.uz0 = float(fz), float(uz0)
    src = list(sources)
    if len(src) > lbd.LBD_MAX_SOURCES:
        raise ValueError("too many sources")
    p.n_src = len(src)
    for k, (x, y, z, R) in enumerate(src):
        p.src[k] = lbd3_source(x, y, z, R)
    return p


def _arr(a, n):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if a.size != n:
        raise ValueError("array has %d elements, expected %d" % (a.size, n))
    return a, a.ctypes.data_as(_dp)


class Sim3:
    """One 3D lattice (nx, ny, nz) on the current device."""

    def __init__(self, nx, ny, nz, precision=lbd.LBD_FP64, sources=(), flags=0, stream=None, **kw):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.params = make_params(precision, sources, flags, **kw)
        g = lbd3_grid(self.nx, self.ny, self.nz)
        self._h = _P()
        rc = load().lbd3_create(ctypes.byref(g), ctypes.byref(self.params),
                                ctypes.c_void_p(stream or 0), ctypes.byref(self._h))
        if rc != lbd.LBD_OK:
            raise lbd.LbdError(rc, "lbd3_create failed")

    def _check(self, rc):
        if rc != lbd.LBD_OK:
            raise lbd.LbdError(rc, load().lbd3_last_error(self._h).decode())

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def set_fields(self, phi, psi, rho=None, u=None):
        u = (None, None, None) if u is None else tuple(u)
        arrs = [_arr(a, self.N) for a in (rho,) + u + (phi, psi)]
        self._check(load().lbd3_set_fields(self._h, *[p for _, p in arrs]))

    def step(self, n=1):
        self._check(load().lbd3_step(self._h, int(n)))
        return self

    @property
    def zrun(self):
        """z planes walked by each CTA of the step kernels."""
        v = ctypes.c_int32()
        self._check(load().lbd3_get_zrun(self._h, ctypes.byref(v)))
        return v.value

    @zrun.setter
    def zrun(self, planes):
        self._check(load().lbd3_set_zrun(self._h, int(planes)))

    def fields(self):
        """(rho, u (3, nz, ny, nx), phi, psi)."""
        out = [np.empty(self.N) for _ in range(6)]
        self._check(load().lbd3_get_fields(self._h, *[o.ctypes.data_as(_dp) for o in out]))
        o = [a.reshape(self.shape) for a in out]
        return o[0], np.stack(o[1:4]), o[4], o[5]

    def populations(self):
        f = np.empty(19 * self.N)
        self._check(load().lbd3_get_populations(self._h, f.ctypes.data_as(_dp)))
        return f.reshape((19,) + self.shape)

    def diagnostics(self, refx, refy, refz):
        d = lbd3_diag()
        self._check(load().lbd3_diagnostics(self._h, float(refx), float(refy), float(refz),
                                            ctypes.byref(d)))
        return {k: getattr(d, k) for k, _ in lbd3_diag._fields_}

    def synchronize(self):
        self._check(load().lbd3_synchronize(self._h))

    @property
    def t(self):
        v = ctypes.c_int64()
        self._check(load().lbd3_get_time(self._h, ctypes.byref(v)))
        return v.value

    def close(self):
        if self._h:
            load().lbd3_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
