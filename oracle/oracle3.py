"""ctypes wrapper of the 3D oracle ``liborc3.so`` (``lbd_oracle3.c``): the
coupled step of Section 2 on the D3Q19 lattice.

TEST INFRASTRUCTURE ONLY (tests/ and the bench's CPU leg).  Arrays are
(nz, ny, nx) float64; populations (19, nz, ny, nx) with the velocity order of
``EX, EY, EZ`` below.
"""
import ctypes

import numpy as np

from . import build as _build

FROZEN_U = 1
BODY_FORCE = 2

EX = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0]
EY = [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1]
EZ = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]

PAPER_PARAMS = dict(a=-0.001, b=0.001, B0=0.006, B1=-0.05, M=1.0, D=0.1, tau=1.0,
                    gamma=0.0, c0=0.0, A0=0.0, A_max=0.0, t_on=0)

_dp = ctypes.POINTER(ctypes.c_double)


class _Params3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)] + \
               [(k, ctypes.c_double) for k in ("a", "b", "B0", "B1", "M", "D", "tau", "gamma",
                                                "c0", "A0", "A_max")] + \
               [("t_on", ctypes.c_int64), ("n_src", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("src", _dp)] + \
               [(k, ctypes.c_double) for k in ("fx", "fy", "fz", "ux0", "uy0", "uz0")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build3())
        P = ctypes.POINTER(_Params3)
        for name, args in [
            ("orc3_grad", [P, _dp, _dp, _dp, _dp]),
            ("orc3_lap", [P, _dp, _dp]),
            ("orc3_force", [P, _dp, _dp, _dp]),
            ("orc3_equilibrium", [ctypes.c_double] * 4 + [_dp]),
            ("orc3_guo", [ctypes.c_double] * 7 + [_dp]),
            ("orc3_run", [P, _dp, _dp, _dp, ctypes.c_int64, ctypes.c_int64]),
            ("orc3_init_equilibrium", [P, _dp, _dp, _dp, _dp, _dp]),
            ("orc3_fields", [P, _dp, _dp, _dp, _dp, _dp]),
        ]:
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = None
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class Params3:
    def __init__(self, nx, ny, nz, sources=(), flags=0, fx=0.0, fy=0.0, fz=0.0, ux0=0.0,
                 uy0=0.0, uz0=0.0, **kw):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.vals = dict(PAPER_PARAMS)
        self.vals.update(kw)
        self.sources = np.ascontiguousarray(np.asarray(sources, dtype=np.float64).reshape(-1, 4))
        self.flags = int(flags)
        self.extra = (fx, fy, fz, ux0, uy0, uz0)

    def c(self):
        v = self.vals
        s = _Params3(self.nx, self.ny, self.nz, *[v[k] for k in ("a", "b", "B0", "B1", "M", "D",
                                                                 "tau", "gamma", "c0", "A0",
                                                                 "A_max")],
                     int(v["t_on"]), len(self.sources), self.flags,
                     self.sources.ctypes.data_as(_dp) if len(self.sources) else None,
                     *self.extra)
        s._keep = self.sources
        return s


class State3:
    """Pre-collision populations and phi, c at time t."""

    def __init__(self, params, phi, psi, rho=None, u=None, t=0):
        self.p = params
        shape = (params.nz, params.ny, params.nx)
        self.phi = np.ascontiguousarray(np.array(phi, dtype=np.float64).reshape(shape))
        self.psi = np.ascontiguousarray(np.array(psi, dtype=np.float64).reshape(shape))
        rho = np.ones(shape) if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        u = np.zeros((3,) + shape) if u is None else np.ascontiguousarray(u, dtype=np.float64)
        self.f = np.zeros((19,) + shape)
        pc = params.c()
        lib().orc3_init_equilibrium(ctypes.byref(pc), _ptr(rho), _ptr(np.ascontiguousarray(u[0])),
                                    _ptr(np.ascontiguousarray(u[1])),
                                    _ptr(np.ascontiguousarray(u[2])), _ptr(self.f))
        self.t = int(t)

    def step(self, n=1):
        pc = self.p.c()
        lib().orc3_run(ctypes.byref(pc), _ptr(self.f), _ptr(self.phi), _ptr(self.psi), self.t,
                       int(n))
        self.t += int(n)
        return self

    def fields(self):
        """(rho, u (3, nz, ny, nx), phi, psi)."""
        shape = self.phi.shape
        rho, u = np.zeros(shape), np.zeros((3,) + shape)
        pc = self.p.c()
        lib().orc3_fields(ctypes.byref(pc), _ptr(self.f), _ptr(self.phi), _ptr(self.psi),
                          _ptr(rho), _ptr(u))
        return rho, u, self.phi.copy(), self.psi.copy()


def grad(params, g):
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = [np.zeros_like(g) for _ in range(3)]
    pc = params.c()
    lib().orc3_grad(ctypes.byref(pc), _ptr(g), *[_ptr(o) for o in out])
    return out


def lap(params, g):
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros_like(g)
    pc = params.c()
    lib().orc3_lap(ctypes.byref(pc), _ptr(g), _ptr(out))
    return out


def equilibrium(n, ux, uy, uz):
    out = np.zeros(19)
    lib().orc3_equilibrium(float(n), float(ux), float(uy), float(uz), _ptr(out))
    return out


def guo(tau, u, F):
    out = np.zeros(19)
    lib().orc3_guo(float(tau), *[float(v) for v in u], *[float(v) for v in F], _ptr(out))
    return out
