"""GPU parity of the FP32 stripe kernel with 16-byte population staging
(launch shapes 116 x by, lbd_vstripe.cu) against the FP64 oracle.

The kernel runs the FP32 form (shifted populations) on periodic lattices whose
width is a multiple of 4.  Tolerances as for the other FP32 kernels: phi, psi
and u within 1e-4 absolute of the oracle, rho within 1e-5, the droplet
centroid within 0.02 lattice units; the three segment lengths of the family
give bit-identical states.
"""
import numpy as np
import pytest

import oracle
from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu

SHAPES = [(116, 32), (116, 64), (116, 128)]
ACTIVE = dict(M=0.5, tau=0.8, gamma=1.5e-3, c0=0.09, A0=1e-6, A_max=1e-4, t_on=20)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    import oracle.build
    oracle.build.build()
    lbd.load()


def droplet(nx, ny, seed, R):
    d = dict(x=nx / 2 - 0.3, y=ny / 2 + 0.4, R=R, psi_mean=0.1, noise=0.01, gx=0.005)
    phi, psi = inputs.droplet_fields(nx, ny, [d], seed=seed)
    return d, phi, psi


def fp32_close(sim, ref):
    g, r = sim.fields(), ref.fields()
    assert np.abs(g[0] - r[0]).max() <= 1e-5
    for k in (1, 2, 3, 4):
        assert np.abs(g[k] - r[k]).max() <= 1e-4, k


@pytest.mark.parametrize("tile", SHAPES, ids=lambda t: "%dx%d" % t)
def test_single_droplet_2000_steps(tile):
    """The 128^2 single-droplet workload (passive, then sink and source ramp)."""
    w = inputs.single_droplet()
    n = w["nx"]
    sim = lbd.Sim(n, n, precision=lbd.LBD_FP32, sources=w["sources"], **w["params"])
    sim.set_tile(*tile)
    sim.set_fields(w["phi"], w["psi"])
    ref = oracle.State(oracle.Params(n, n, sources=w["sources"], **w["params"]), w["phi"], w["psi"])
    for _ in range(4):
        sim.step(500)
        ref.step(500)
        fp32_close(sim, ref)
        dg, dr = sim.diagnostics(64, 64), ref.diagnostics(64, 64)
        assert abs(dg["cm_x"] - dr["cm_x"]) <= 0.02 and abs(dg["cm_y"] - dr["cm_y"]) <= 0.02


@pytest.mark.parametrize("tile", SHAPES, ids=lambda t: "%dx%d" % t)
@pytest.mark.parametrize("nx,ny", [(100, 37), (8, 8), (4, 5), (236, 41), (300, 130), (464, 23)])
def test_ragged_and_small_grids(nx, ny, tile):
    """Lattices spanning several stripes with a ragged last stripe (236 = 2 x 116
    + 4), a segment tail, and lattices narrower than one window (the 136-column
    staging window wraps the periodic seam several times)."""
    d, phi, psi = droplet(nx, ny, seed=nx * 1000 + ny, R=max(1.5, min(nx, ny) / 4))
    src = [(nx / 3, ny / 2, max(1.0, min(nx, ny) / 8))]
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP32, sources=src, **ACTIVE)
    sim.set_tile(*tile)
    sim.set_fields(phi, psi)
    sim.step(150)
    ref = oracle.State(oracle.Params(nx, ny, sources=src, **ACTIVE), phi, psi).step(150)
    fp32_close(sim, ref)


def test_shapes_bit_identical_and_agree_with_stripe_kernel():
    nx, ny = 348, 70
    d, phi, psi = droplet(nx, ny, seed=5, R=17.0)
    src = [inputs.default_source(d, nx, ny)]
    outs = []
    for t in SHAPES + [(118, 64)]:
        sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP32, sources=src, **ACTIVE)
        sim.set_tile(*t)
        sim.set_fields(phi, psi)
        sim.step(60)
        outs.append((sim.fields(), sim.populations()))
    for o in outs[1:3]:
        for a, b in zip(o[0], outs[0][0]):
            assert np.array_equal(a, b)
        assert np.array_equal(o[1], outs[0][1])
    for a, b in zip(outs[0][0], outs[3][0]):
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(b).max(), 1e-3)


def test_rejected_where_unsupported():
    for nx, prec, flags in [(102, lbd.LBD_FP32, 0), (128, lbd.LBD_FP64, 0),
                            (128, lbd.LBD_FP32, lbd.LBD_WALLS)]:
        sim = lbd.Sim(nx, 16, precision=prec, flags=flags)
        with pytest.raises(lbd.LbdError) as e:
            sim.set_tile(116, 64)
        assert e.value.code == lbd.LBD_EINVAL
        sim.close()


def test_body_force_and_frozen_velocity():
    """The flag paths of the kernel: a uniform body force adds exactly N F of
    momentum per step; a frozen velocity field advects phi and psi as in the
    oracle."""
    nx, ny = 40, 36
    F = (1e-5, -2e-5)
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP32, flags=lbd.LBD_BODY_FORCE, fx=F[0], fy=F[1])
    sim.set_tile(116, 32)
    sim.set_fields(np.full((ny, nx), 0.9), np.full((ny, nx), 0.1))
    sim.step(25)
    f = sim.populations()
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    assert np.einsum("iyx,i->", f, ex) == pytest.approx(F[0] * 25 * nx * ny, rel=1e-4)
    assert np.einsum("iyx,i->", f, ey) == pytest.approx(F[1] * 25 * nx * ny, rel=1e-4)
    d, phi, psi = droplet(nx, ny, seed=2, R=9.0)
    kw = dict(ux0=0.05, uy0=-0.03, M=0.3)
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP32, flags=lbd.LBD_FROZEN_U, **kw)
    sim.set_tile(116, 32)
    sim.set_fields(phi, psi)
    sim.step(100)
    ref = oracle.State(oracle.Params(nx, ny, flags=lbd.LBD_FROZEN_U, **kw), phi, psi).step(100)
    g, r = sim.fields(), ref.fields()
    for k in (3, 4):
        assert np.abs(g[k] - r[k]).max() <= 1e-4, k
