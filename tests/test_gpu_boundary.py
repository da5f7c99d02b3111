"""GPU checks of two boundary calls: the seeded device-side initial state
(lbd_init_droplets) against the host generator it restates
(inputs.droplet_fields, same SplitMix64 stream), and the device read-back
(lbd_get_fields_device) against the host read-back."""
import numpy as np
import pytest

from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu

DROPS = [dict(x=20.3, y=30.7, R=12.0, psi_mean=0.1, noise=0.01, gx=0.004, gy=-0.002),
         dict(x=95.5, y=2.0, R=9.0, psi_mean=0.11, noise=0.005),   # wraps through y = 0
         dict(x=1.0, y=70.0, R=15.0, noise=0.008, gx=-0.003)]      # wraps through x = 0


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    lbd.load()


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("seed", [7, 2 ** 63 + 12345])
def test_init_droplets_matches_host_generator(prec, seed):
    nx, ny = 128, 96
    phi, psi = inputs.droplet_fields(nx, ny, DROPS, seed=seed)
    a = lbd.Sim(nx, ny, precision=prec)
    a.init_droplets(DROPS, psi_bg=0.1, seed=seed)
    g = a.fields()
    tol = 4e-15 if prec == lbd.LBD_FP64 else 1e-7  # a few ulps of tanh and sqrt
    assert np.abs(g[3] - phi).max() <= tol
    assert np.abs(g[4] - psi).max() <= tol
    # at rest: the same density and velocity (u = F / 2n from the same force) as
    # the state uploaded from the host generator, and the states evolve alike
    b = lbd.Sim(nx, ny, precision=prec)
    b.set_fields(phi, psi)
    h = b.fields()
    assert np.abs(g[0] - 1.0).max() == 0.0
    for k in (1, 2):
        assert np.abs(g[k] - h[k]).max() <= (1e-13 if prec == lbd.LBD_FP64 else 1e-6) * max(
            np.abs(h[k]).max(), 1e-12)
    a.step(50)
    b.step(50)
    ga, gb = a.fields(), b.fields()
    for x, y in zip(ga, gb):
        assert np.abs(x - y).max() <= (1e-13 if prec == lbd.LBD_FP64 else 1e-5)
    a.close()
    b.close()


def test_init_droplets_rejects_unstable_psi():
    s = lbd.Sim(64, 64, precision=lbd.LBD_FP64)
    with pytest.raises(lbd.LbdError) as e:
        s.init_droplets([dict(x=32, y=32, R=10, psi_mean=0.01, noise=0.02)])
    assert e.value.code == lbd.LBD_EUNSTABLE
    with pytest.raises(lbd.LbdError) as e:
        s.init_droplets([dict(x=32, y=32, R=10, psi_mean=0.2)])  # B = 0.006 - 0.05 * 0.2 < 0
    assert e.value.code == lbd.LBD_EUNSTABLE
    s.close()


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32], ids=["fp64", "fp32"])
def test_fields_device_equals_host_read_back(prec):
    torch = pytest.importorskip("torch")
    nx, ny = 100, 60
    s = lbd.Sim(nx, ny, precision=prec, M=0.5, tau=0.8)
    s.init_droplets(DROPS[:1], seed=3)
    s.step(30)
    host = s.fields()
    dt = torch.float64 if prec == lbd.LBD_FP64 else torch.float32
    outs = [torch.full((ny, nx), float("nan"), dtype=dt, device="cuda") for _ in range(5)]
    s.fields_device(*[t.data_ptr() for t in outs])
    s.synchronize()
    for h, d in zip(host, outs):
        assert np.array_equal(d.cpu().numpy(), h.astype(d.cpu().numpy().dtype))
    # NULL outputs are skipped
    skip = torch.full((ny, nx), -7.0, dtype=dt, device="cuda")
    s.fields_device(0, 0, 0, skip.data_ptr(), 0)
    s.synchronize()
    assert np.array_equal(skip.cpu().numpy(), host[3].astype(skip.cpu().numpy().dtype))
    s.close()


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("flags", [0, lbd.LBD_WALLS], ids=["periodic", "plates"])
def test_checkpoint_restart(prec, flags):
    """Resume from (phi, psi, f, t) read back mid-run: the resumed run follows the
    uninterrupted one (FP32 bitwise; FP64 to the rounding of f - w)."""
    nx, ny = 128, 64
    kw = dict(M=0.5, tau=0.8, gamma=1.5e-3, c0=0.09, A0=1e-6, A_max=1e-4, t_on=30)
    src = [(60.0, 30.0, 3.0)]
    a = lbd.Sim(nx, ny, precision=prec, sources=src, flags=flags, **kw)
    a.init_droplets([dict(x=60.0, y=30.0, R=14.0, noise=0.01, gx=0.005)], seed=9)
    a.step(70)
    _, _, _, phi, psi = a.fields()
    f, t = a.populations(), a.t
    b = lbd.Sim(nx, ny, precision=prec, sources=src, flags=flags, **kw)
    b.set_fields(phi, psi)
    b.set_populations(f)
    b.t = t
    assert np.array_equal(b.populations(), f) if prec == lbd.LBD_FP32 else \
        np.abs(b.populations() - f).max() <= 1e-16
    a.step(100)
    b.step(100)
    for x, y in zip(a.fields(), b.fields()):
        if prec == lbd.LBD_FP32:
            assert np.array_equal(x, y)
        else:
            assert np.abs(x - y).max() <= 1e-13 * max(np.abs(x).max(), 1e-3)
    a.close()
    b.close()
