"""GPU parity of the 3D (D3Q19) coupled step (include/lbd3.h) against the 3D
FP64 oracle, which is itself pinned to the 2D oracle by its exact reduction for
z-invariant states.

Tolerances as in 2D: FP64 max relative error <= 1e-10 per field and for the
populations; FP32 (shifted populations) phi, psi, u within 1e-4 absolute.
"""
import numpy as np
import pytest

from oracle import oracle3 as O3
from paper_1711_10984_gb300 import inputs, lbd, lbd3

pytestmark = pytest.mark.gpu

ACTIVE = dict(M=0.5, tau=0.8, gamma=1.5e-3, c0=0.09, A0=1e-6, A_max=1e-4, t_on=20, B1=-0.03)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    import oracle.build
    oracle.build.build()
    lbd3.load()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def case(nx, ny, nz, seed):
    R = max(2.0, min(nx, ny, nz) / 3)
    c = (nx / 2 - 0.3, ny / 2 + 0.4, nz / 2 - 0.2)
    phi, psi = inputs.sphere_fields(nx, ny, nz, [c + (R,)], B1=ACTIVE["B1"], noise=0.01,
                                    seed=seed)
    src = [(c[0] + R / 2, c[1], c[2], max(1.0, R / 3))]
    return phi, psi, src


def run_both(nx, ny, nz, steps, prec, seed, flags=0, **kw):
    phi, psi, src = case(nx, ny, nz, seed)
    par = dict(ACTIVE, **kw)
    sim = lbd3.Sim3(nx, ny, nz, precision=prec, sources=src, flags=flags, **par)
    sim.set_fields(phi, psi)
    sim.step(steps)
    ref = O3.State3(O3.Params3(nx, ny, nz, sources=src, flags=flags, **par), phi, psi).step(steps)
    return sim, ref


@pytest.mark.parametrize("nx,ny,nz", [(24, 20, 16), (17, 9, 5), (33, 7, 3), (8, 8, 1)])
def test_fp64_3d_matches_oracle(nx, ny, nz):
    sim, ref = run_both(nx, ny, nz, 120, lbd.LBD_FP64, seed=nx + ny + nz)
    r, u, ph, ps = sim.fields()
    r2, u2, ph2, ps2 = ref.fields()
    for a, b in ((r, r2), (u, u2), (ph, ph2), (ps, ps2)):
        assert rel(a, b) <= 1e-10
    assert rel(sim.populations(), ref.f) <= 1e-10
    sim.close()


@pytest.mark.parametrize("flags,kw", [(lbd.LBD_BODY_FORCE, dict(fx=2e-5, fy=-1e-5, fz=3e-5)),
                                      (lbd.LBD_FROZEN_U, dict(ux0=0.02, uy0=-0.01, uz0=0.015))])
def test_fp64_3d_flags(flags, kw):
    sim, ref = run_both(16, 12, 10, 80, lbd.LBD_FP64, seed=4, flags=flags, **kw)
    r, u, ph, ps = sim.fields()
    r2, u2, ph2, ps2 = ref.fields()
    for a, b in ((r, r2), (u, u2), (ph, ph2), (ps, ps2)):
        assert rel(a, b) <= 1e-10
    sim.close()


def test_fp32_3d_tolerance():
    sim, ref = run_both(32, 32, 32, 300, lbd.LBD_FP32, seed=7)
    r, u, ph, ps = sim.fields()
    r2, u2, ph2, ps2 = ref.fields()
    assert np.abs(u - u2).max() <= 1e-4
    assert np.abs(ph - ph2).max() <= 1e-4
    assert np.abs(ps - ps2).max() <= 1e-4
    sim.close()


def test_z_invariant_3d_equals_2d_gpu():
    """nz = 1 with z-invariant fields: the 3D GPU step equals the 2D GPU step."""
    nx, ny = 40, 36
    d = dict(x=19.7, y=18.4, R=10.0, psi_mean=0.1, noise=0.01, gx=0.005)
    phi, psi = inputs.droplet_fields(nx, ny, [d], seed=2)
    kw = dict(ACTIVE)
    s2 = lbd.Sim(nx, ny, precision=lbd.LBD_FP64, sources=[(24.0, 18.0, 3.0)], **kw)
    s2.set_tile(118, 64)
    s2.set_fields(phi, psi)
    s2.step(150)
    s3 = lbd3.Sim3(nx, ny, 1, precision=lbd.LBD_FP64, sources=[(24.0, 18.0, 0.0, 3.0)], **kw)
    s3.set_fields(phi[None], psi[None])
    s3.step(150)
    g2, g3 = s2.fields(), s3.fields()
    assert rel(g3[2][0], g2[3]) <= 1e-11   # phi
    assert rel(g3[3][0], g2[4]) <= 1e-11   # psi
    assert rel(g3[1][0, 0], g2[1]) <= 1e-10  # ux
    assert np.abs(g3[1][2]).max() <= 1e-15  # +-z populations cancel to rounding
    s2.close()
    s3.close()


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32], ids=["fp64", "fp32"])
def test_3d_conservation_and_diagnostics(prec):
    n = 48
    phi, psi = inputs.sphere_fields(n, n, n, [(20.0, 24.0, 26.0, 10.0)], noise=0.01, seed=1)
    sim = lbd3.Sim3(n, n, n, precision=prec, M=0.5, tau=0.8, B1=-0.03)
    sim.set_fields(phi, psi)
    d0 = sim.diagnostics(20, 24, 26)
    assert d0["cm_x"] == pytest.approx(20.0, abs=0.05)
    sim.step(500)
    d1 = sim.diagnostics(20, 24, 26)
    tol = 1e-12 if prec == lbd.LBD_FP64 else 1e-5
    for k in ("sum_rho", "sum_phi", "sum_psi"):
        assert abs(d1[k] - d0[k]) <= tol * abs(d0[k]), k
    assert d1["nonfinite"] == 0
    sim.close()


def test_3d_rejects_bad_fields():
    sim = lbd3.Sim3(8, 8, 8, precision=lbd.LBD_FP64)
    z = np.zeros((8, 8, 8))
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields(z, np.full((8, 8, 8), -0.1))
    assert e.value.code == lbd.LBD_EUNSTABLE
    bad = z.copy()
    bad[1, 2, 3] = np.nan
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields(bad, np.full((8, 8, 8), 0.1))
    assert e.value.code == lbd.LBD_ENONFINITE
    assert "site %d" % ((1 * 8 + 2) * 8 + 3) in str(e.value)
    rho = np.ones((8, 8, 8))
    rho[0, 0, 5] = -1.0
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields(z, np.full((8, 8, 8), 0.1), rho=rho)
    assert e.value.code == lbd.LBD_EINVAL
    # a rejected upload leaves the state as it was
    good = np.tanh(np.linspace(-2, 2, 8))[None, None, :].repeat(8, 0).repeat(8, 1)
    sim.set_fields(good, np.full((8, 8, 8), 0.1))
    before = sim.fields()
    with pytest.raises(lbd.LbdError):
        sim.set_fields(bad, np.full((8, 8, 8), 0.1))
    for a, b in zip(sim.fields(), before):
        assert np.array_equal(a, b)
    sim.close()


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32], ids=["fp64", "fp32"])
def test_3d_zrun_does_not_change_results(prec):
    """Every run length of the z-marching kernels gives bit-identical states,
    including runs of one plane and a ragged last run."""
    nx, ny, nz = 40, 20, 19
    phi, psi, src = case(nx, ny, nz, seed=3)
    outs = []
    for zl in (0, 1, 3, 7, 19):
        sim = lbd3.Sim3(nx, ny, nz, precision=prec, sources=src, **ACTIVE)
        if zl:
            sim.zrun = zl
        assert sim.zrun == zl or zl == 0
        sim.set_fields(phi, psi)
        sim.step(40)
        outs.append((sim.populations(), sim.fields()))
        sim.close()
    for f, fl in outs[1:]:
        assert np.array_equal(f, outs[0][0])
        for a, b in zip(fl, outs[0][1]):
            assert np.array_equal(a, b)


def test_3d_zrun_rejects_out_of_range():
    sim = lbd3.Sim3(8, 8, 6, precision=lbd.LBD_FP32)
    auto = sim.zrun
    assert 1 <= auto <= 6
    for bad in (-1, 7):
        with pytest.raises(lbd.LbdError) as e:
            sim.zrun = bad
        assert e.value.code == lbd.LBD_EINVAL
    sim.zrun = 6
    sim.zrun = 0
    assert sim.zrun == auto
    sim.close()


def test_fp32_3d_full_size():
    """The bench's 3D workload at full size: 256^3, 64 droplets R = 16 with a
    source ball each, in the launch shape the bench times (automatic z runs).
    The GPU state after 40 steps (populations, phi, psi, t) is handed to the 3D
    oracle; after 2 more steps on both, phi, psi and u agree within 1e-4 over the
    whole box."""
    n = 256
    w = inputs.emulsion3(n=n)
    sim = lbd3.Sim3(n, n, n, precision=lbd.LBD_FP32, sources=w["sources"], **w["params"])
    sim.set_fields(w["phi"], w["psi"])
    sim.step(40)
    _, _, phi, psi = sim.fields()
    ref = O3.State3(O3.Params3(n, n, n, sources=w["sources"], **w["params"]), phi, psi, t=40)
    ref.f[...] = sim.populations()
    sim.step(2)
    ref.step(2)
    _, u, ph, ps = sim.fields()
    _, u2, ph2, ps2 = ref.fields()
    sim.close()
    assert np.abs(u - u2).max() <= 1e-4
    assert np.abs(ph - ph2).max() <= 1e-4
    assert np.abs(ps - ps2).max() <= 1e-4
    assert np.abs(u2).max() > 0
