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


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
def test_static_scratch_diagnostics_match(prec):
    torch = pytest.importorskip("torch")
    nx, ny = 200, 150
    d = dict(x=90.5, y=70.0, R=30.0, psi_mean=0.1, noise=0.01, gx=0.005)
    phi, psi = inputs.droplet_fields(nx, ny, [d], seed=21)
    kw = dict(M=0.5, tau=0.8, gamma=1.5e-3, c0=0.09, A0=1e-6, A_max=1e-4, t_on=0)
    src = [inputs.default_source(d, nx, ny)]
    sim = lbd.Sim(nx, ny, precision=prec, sources=src, **kw)
    sim.set_fields(phi, psi)
    sim.step(120)

    # the same state, copied into device buffers that the test owns
    f = sim.populations()
    _, _, _, ph, ps = sim.fields()
    dt = torch.float64 if prec == lbd.LBD_FP64 else torch.float32
    g_dev = torch.tensor(f - W[:, None, None], dtype=dt, device="cuda").contiguous()
    phi_dev = torch.tensor(ph, dtype=dt, device="cuda").contiguous()
    psi_dev = torch.tensor(ps, dtype=dt, device="cuda").contiguous()
    torch.cuda.synchronize()

    L = lbd.load()
    for refx, refy in [(d["x"], d["y"]), (5.0, 140.0)]:
        want = sim.diagnostics(refx, refy)
        for call in range(2):
            out = lbd.lbd_diag()
            rc = L.lbd_diagnostics_static(nx, ny, nx, prec, g_dev.data_ptr(), phi_dev.data_ptr(),
                                          psi_dev.data_ptr(), kw.get("B0", 0.006),
                                          kw.get("B1", -0.05), refx, refy, None,
                                          ctypes.byref(out))
            assert rc == lbd.LBD_OK, (call, rc)
            got = {k: getattr(out, k) for k, _ in lbd.lbd_diag._fields_}
            tol = 1e-12 if prec == lbd.LBD_FP64 else 1e-7
            for k in ("sum_rho", "sum_phi", "sum_psi", "mass_pos"):
                assert abs(got[k] - want[k]) <= tol * max(abs(want[k]), 1.0), (call, k)
            ctol = 1e-10 if prec == lbd.LBD_FP64 else 1e-5
            assert abs(got["cm_x"] - want["cm_x"]) <= ctol, call
            assert abs(got["cm_y"] - want["cm_y"]) <= ctol, call
            assert got["min_B"] == want["min_B"] and got["min_psi"] == want["min_psi"]
            assert got["nonfinite"] == want["nonfinite"] == 0
    sim.close()


def test_static_scratch_rejects_oversized_lattice():
    out = lbd.lbd_diag()
    L = lbd.load()
    big = (1 << 20) + 1
    rc = L.lbd_diagnostics_static(big, 8, big, lbd.LBD_FP64, 1, 1, 1, 0.006, -0.05, 0.0, 0.0,
                                  None, ctypes.byref(out))
    assert rc == lbd.LBD_EINVAL
