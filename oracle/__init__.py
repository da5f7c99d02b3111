"""FP64 CPU oracle of the coupled LB/FD step (arXiv 1711.10984, Section 2).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``, never by the product package.  Two
independent restatements live here:

* ``liborc.so`` (``lbd_oracle.c``): plain per-site C loops, the primary oracle;
* ``torch_ref`` : a vectorised ``torch.roll`` restatement in float64, written
  separately, used to cross-check the C oracle and as the reverse-mode
  (autograd) reference for the adjoint.

Parity status per function (pins in ``tests/test_oracle_*.py``):
  stencils, equilibrium, Guo forcing, advection, diffusion, source/sink,
  conservation, flat-interface profile, Laplace law, shear-wave decay,
  Galilean invariance, free-energy density (Table 1 sigma_num); walls (Poiseuille
  profile, conservation, mirror equivalence of the FD part): pinned.  The full nonlinear coupled trajectory has no
  printed values to compare with; it is pinned only through the invariants and
  the agreement of the two restatements.
"""
import ctypes
import os

import numpy as np

from . import build as _build

FROZEN_U = 1
BODY_FORCE = 2
LITERAL_ADVECTION = 4
LITERAL_LOG = 8
WALLS = 16   # bounce-back plates at y = -1/2 and y = ny - 1/2 (C oracle only)

# Section 2.1 / 3 parameter set used throughout the paper's equilibrium tests.
PAPER_PARAMS = dict(a=-0.001, b=0.001, B0=0.006, B1=-0.05, M=1.0, D=0.1, tau=1.0,
                    gamma=0.0, c0=0.0, A0=0.0, A_max=0.0, t_on=0)

_dp = ctypes.POINTER(ctypes.c_double)


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("B0", ctypes.c_double), ("B1", ctypes.c_double),
                ("M", ctypes.c_double), ("D", ctypes.c_double), ("tau", ctypes.c_double),
                ("gamma", ctypes.c_double), ("c0", ctypes.c_double),
                ("A0", ctypes.c_double), ("A_max", ctypes.c_double),
                ("t_on", ctypes.c_int64), ("n_src", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("src", _dp), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("ux0", ctypes.c_double), ("uy0", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        P = ctypes.POINTER(_Params)
        for name, args in [
            ("orc_grad", [P, _dp, _dp, _dp]),
            ("orc_lap", [P, _dp, _dp]),
            ("orc_force", [P, _dp, _dp, _dp, _dp]),
            ("orc_equilibrium", [ctypes.c_double] * 3 + [_dp]),
            ("orc_guo", [ctypes.c_double] * 5 + [_dp]),
            ("orc_moments", [P, _dp, _dp, _dp, _dp, _dp, _dp]),
            ("orc_step", [P, _dp, _dp, _dp, ctypes.c_int64]),
            ("orc_run", [P, _dp, _dp, _dp, ctypes.c_int64, ctypes.c_int64]),
            ("orc_fields", [P, _dp, _dp, _dp, _dp, _dp, _dp]),
            ("orc_init_equilibrium", [P, _dp, _dp, _dp, _dp]),
            ("orc_pressure", [P, _dp, _dp, _dp, _dp]),
            ("orc_free_energy", [P, _dp, _dp, _dp]),
            ("orc_diagnostics", [P, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
            ("orc_activity", [P, ctypes.c_int64, _dp, _dp]),
        ]:
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = None
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class Params:
    """Plain parameter holder: dict of the model parameters + grid + sources."""

    def __init__(self, nx, ny, sources=(), flags=0, fx=0.0, fy=0.0, ux0=0.0, uy0=0.0, **kw):
        self.nx, self.ny = int(nx), int(ny)
        vals = dict(PAPER_PARAMS)
        vals.update(kw)
        self.vals = vals
        self.sources = np.ascontiguousarray(np.asarray(sources, dtype=np.float64).reshape(-1, 3))
        self.flags, self.fx, self.fy, self.ux0, self.uy0 = int(flags), fx, fy, ux0, uy0

    def c(self):
        v = self.vals
        s = _Params(self.nx, self.ny, v["a"], v["b"], v["B0"], v["B1"], v["M"], v["D"],
                    v["tau"], v["gamma"], v["c0"], v["A0"], v["A_max"], int(v["t_on"]),
                    len(self.sources), self.flags,
                    self.sources.ctypes.data_as(_dp) if len(self.sources) else None,
                    self.fx, self.fy, self.ux0, self.uy0)
        s._keep = self.sources
        return s

    def __getitem__(self, k):
        return self.vals[k]


class State:
    """Pre-collision populations f (9, ny, nx) and phi, c (ny, nx) at time t."""

    def __init__(self, params, phi, psi, rho=None, ux=None, uy=None, t=0):
        self.p = params
        shape = (params.ny, params.nx)
        self.phi = np.ascontiguousarray(np.array(phi, dtype=np.float64).reshape(shape))
        self.psi = np.ascontiguousarray(np.array(psi, dtype=np.float64).reshape(shape))
        rho = np.ones(shape) if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        ux = np.zeros(shape) if ux is None else np.ascontiguousarray(ux, dtype=np.float64)
        uy = np.zeros(shape) if uy is None else np.ascontiguousarray(uy, dtype=np.float64)
        self.f = np.zeros((9,) + shape)
        pc = params.c()
        lib().orc_init_equilibrium(ctypes.byref(pc), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(self.f))
        self.t = int(t)

    def step(self, n=1):
        pc = self.p.c()
        lib().orc_run(ctypes.byref(pc), _ptr(self.f), _ptr(self.phi), _ptr(self.psi), self.t, int(n))
        self.t += int(n)
        return self

    def fields(self):
        """(rho, ux, uy, phi, psi) at the current time, u from Eq. (11)."""
        shape = self.phi.shape
        rho, ux, uy = np.zeros(shape), np.zeros(shape), np.zeros(shape)
        pc = self.p.c()
        lib().orc_fields(ctypes.byref(pc), _ptr(self.f), _ptr(self.phi), _ptr(self.psi),
                         _ptr(rho), _ptr(ux), _ptr(uy))
        return rho, ux, uy, self.phi.copy(), self.psi.copy()

    def diagnostics(self, refx, refy):
        out = np.zeros(9)
        pc = self.p.c()
        lib().orc_diagnostics(ctypes.byref(pc), _ptr(self.f), _ptr(self.phi), _ptr(self.psi),
                              float(refx), float(refy), _ptr(out))
        keys = ["sum_rho", "sum_phi", "sum_psi", "cm_x", "cm_y", "min_B", "min_psi",
                "nonfinite", "mass_pos"]
        return dict(zip(keys, out.tolist()))

    def pressure(self):
        rho = self.fields()[0]
        p0 = np.zeros_like(rho)
        pc = self.p.c()
        lib().orc_pressure(ctypes.byref(pc), _ptr(rho), _ptr(self.phi), _ptr(self.psi), _ptr(p0))
        return p0


def grad(params, g):
    g = np.ascontiguousarray(g, dtype=np.float64)
    gx, gy = np.zeros_like(g), np.zeros_like(g)
    pc = params.c()
    lib().orc_grad(ctypes.byref(pc), _ptr(g), _ptr(gx), _ptr(gy))
    return gx, gy


def lap(params, g):
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros_like(g)
    pc = params.c()
    lib().orc_lap(ctypes.byref(pc), _ptr(g), _ptr(out))
    return out


def force(params, phi, psi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    Fx, Fy = np.zeros_like(phi), np.zeros_like(phi)
    pc = params.c()
    lib().orc_force(ctypes.byref(pc), _ptr(phi), _ptr(psi), _ptr(Fx), _ptr(Fy))
    return Fx, Fy


def equilibrium(n, ux, uy):
    out = np.zeros(9)
    lib().orc_equilibrium(float(n), float(ux), float(uy), _ptr(out))
    return out


def guo(tau, ux, uy, Fx, Fy):
    out = np.zeros(9)
    lib().orc_guo(float(tau), float(ux), float(uy), float(Fx), float(Fy), _ptr(out))
    return out


def free_energy(params, phi, psi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    out = np.zeros_like(phi)
    pc = params.c()
    lib().orc_free_energy(ctypes.byref(pc), _ptr(phi), _ptr(psi), _ptr(out))
    return out


def activity(params, t):
    A, g = ctypes.c_double(), ctypes.c_double()
    pc = params.c()
    lib().orc_activity(ctypes.byref(pc), int(t), ctypes.byref(A), ctypes.byref(g))
    return A.value, g.value
