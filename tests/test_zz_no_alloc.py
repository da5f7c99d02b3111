"""lbd_diagnostics_static: diagnostics without any device allocation.

Some callers cannot call cudaMalloc: their device memory all comes from another
allocator (a framework's caching pool, an arena reserved at start-up), or their
loops must not pay the device synchronisation that cudaMalloc/cudaFree can
cause.  For them the library offers lbd_diagnostics_static, which takes the
state in the caller's own device buffers and does its reduction in a fixed
scratch array compiled into the library.  This test holds its result to the
one of lbd_diagnostics (which uses scratch allocated by lbd_create) on the same
state, within the tolerances of the other diagnostics tests, on two calls in a
row (the second call reuses the scratch the first one left behind).

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    lbd.load()


def _state(prec, nx, ny, seed, steps, R):
    d = dict(x=nx * 0.45 + 0.5, y=ny * 0.47, R=R, psi_mean=0.1, noise=0.01, gx=0.005)
    phi, psi = inputs.droplet_fields(nx, ny, [d], seed=seed)
    kw = dict(M=0.5, tau=0.8, gamma=1.5e-3, c0=0.09, A0=1e-6, A_max=1e-4, t_on=0)
    sim = lbd.Sim(nx, ny, precision=prec, sources=[inputs.default_source(d, nx, ny)], **kw)
    sim.set_fields(phi, psi)
    sim.step(steps)
    return sim, d


def _device_copy(torch, sim, prec, pad):
    """The state of sim in device buffers owned by the test, rows padded by pad
    elements (pitch = nx + pad); returns the three buffers and the pitch."""
    f = sim.populations()
    _, _, _, ph, ps = sim.fields()
    dt = torch.float64 if prec == lbd.LBD_FP64 else torch.float32
    ny, nx = ph.shape
    pitch = nx + pad
    g = torch.full((9, ny, pitch), float("nan"), dtype=dt, device="cuda")
    p1 = torch.full((ny, pitch), float("nan"), dtype=dt, device="cuda")
    p2 = torch.full((ny, pitch), float("nan"), dtype=dt, device="cuda")
    g[:, :, :nx] = torch.tensor(f - W[:, None, None], dtype=dt)
    p1[:, :nx] = torch.tensor(ph, dtype=dt)
    p2[:, :nx] = torch.tensor(ps, dtype=dt)
    return (g, p1, p2), pitch


def _call(L, nx, ny, pitch, prec, bufs, refx, refy, stream):
    out = lbd.lbd_diag()
    rc = L.lbd_diagnostics_static(nx, ny, pitch, prec, bufs[0].data_ptr(), bufs[1].data_ptr(),
                                  bufs[2].data_ptr(), 0.006, -0.05, refx, refy, stream,
                                  ctypes.byref(out))
    assert rc == lbd.LBD_OK, rc
    return {k: getattr(out, k) for k, _ in lbd.lbd_diag._fields_}


def _agree(got, want, prec, what):
    tol = 1e-12 if prec == lbd.LBD_FP64 else 1e-7
    for k in ("sum_rho", "sum_phi", "sum_psi", "mass_pos"):
        assert abs(got[k] - want[k]) <= tol * max(abs(want[k]), 1.0), (what, k)
    ctol = 1e-10 if prec == lbd.LBD_FP64 else 1e-5
    assert abs(got["cm_x"] - want["cm_x"]) <= ctol, what
    assert abs(got["cm_y"] - want["cm_y"]) <= ctol, what
    assert got["min_B"] == want["min_B"] and got["min_psi"] == want["min_psi"], what
    assert got["nonfinite"] == want["nonfinite"] == 0, what


@pytest.mark.parametrize("pad", [0, 24], ids=["pitch=nx", "pitch=nx+24"])
@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
def test_static_scratch_diagnostics_match(prec, pad):
    """Two calls in a row on the same state agree with lbd_diagnostics, also with
    a call on a different (smaller) lattice in the other precision between
    them, whose own results must not leak into the next call's (both forms
    share the one scratch array); on the legacy stream and on a caller-given
    stream; with unpadded and padded rows (the padding is NaN, so a read of it
    would show)."""
    torch = pytest.importorskip("torch")
    nx, ny = 200, 150
    oprec = lbd.LBD_FP32 if prec == lbd.LBD_FP64 else lbd.LBD_FP64
    sim, d = _state(prec, nx, ny, seed=21, steps=120, R=30.0)
    other, od = _state(oprec, 72, 40, seed=5, steps=30, R=12.0)
    bufs, pitch = _device_copy(torch, sim, prec, pad)
    obufs, opitch = _device_copy(torch, other, oprec, 8)
    torch.cuda.synchronize()
    L = lbd.load()
    side = torch.cuda.Stream()
    for stream in (None, side.cuda_stream):
        for refx, refy in [(d["x"], d["y"]), (5.0, 140.0)]:
            want = sim.diagnostics(refx, refy)
            got1 = _call(L, nx, ny, pitch, prec, bufs, refx, refy, stream)
            _agree(got1, want, prec, "first call")
            owant = other.diagnostics(od["x"], od["y"])
            ogot = _call(L, 72, 40, opitch, oprec, obufs, od["x"], od["y"], stream)
            _agree(ogot, owant, oprec, "other lattice")
            got2 = _call(L, nx, ny, pitch, prec, bufs, refx, refy, stream)
            _agree(got2, want, prec, "second call")
    sim.close()
    other.close()


def test_static_scratch_rejects_host_pointer():
    """A host buffer handed in where device memory belongs is refused
    (LBD_EINVAL) instead of reaching the kernel."""
    torch = pytest.importorskip("torch")
    nx, ny = 16, 8
    host = np.zeros(9 * nx * ny)
    dev = torch.zeros(9 * nx * ny, dtype=torch.float64, device="cuda")
    L = lbd.load()
    out = lbd.lbd_diag()
    hp = host.ctypes.data
    for g, phi, psi in ((hp, dev.data_ptr(), dev.data_ptr()),
                        (dev.data_ptr(), hp, dev.data_ptr()),
                        (dev.data_ptr(), dev.data_ptr(), hp)):
        rc = L.lbd_diagnostics_static(nx, ny, nx, lbd.LBD_FP64, g, phi, psi, 0.006, -0.05, 1.0,
                                      1.0, None, ctypes.byref(out))
        assert rc == lbd.LBD_EINVAL


def test_static_scratch_rejects_oversized_lattice():
    out = lbd.lbd_diag()
    L = lbd.load()
    big = (1 << 20) + 1
    rc = L.lbd_diagnostics_static(big, 8, big, lbd.LBD_FP64, 1, 1, 1, 0.006, -0.05, 0.0, 0.0,
                                  None, ctypes.byref(out))
    assert rc == lbd.LBD_EINVAL
