"""GPU parity with walls (LBD_WALLS: bounce-back plates at y = -1/2 and
y = ny - 1/2, mirrored finite-difference fields, no advective flux through a
plate) against the FP64 oracle with the same reading.

Tolerances as for the periodic lattice: FP64 max relative error <= 1e-10 per
field and for the populations; FP32 (shifted populations) phi, psi, u within
1e-4 absolute.
"""
import numpy as np
import pytest

import oracle
from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu

ACTIVE = dict(M=0.5, tau=0.8, gamma=1.5e-3, c0=0.09, A0=1e-6, A_max=1e-4, t_on=20)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    import oracle.build
    oracle.build.build()
    lbd.load()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def wall_droplet(nx, ny, seed):
    """A droplet whose interface reaches the bottom plate, a source inside it
    next to the plate, and seeded noise everywhere."""
    R = max(3.0, min(nx, ny) / 3)
    d = dict(x=nx / 2 - 0.3, y=R - 1.5, R=R, psi_mean=0.1, noise=0.01, gx=0.005)
    phi, psi = inputs.droplet_fields(nx, ny, [d], seed=seed)
    src = [(nx / 2 + R / 3, 1.0, max(1.0, R / 3))]
    return phi, psi, src


def run_both(nx, ny, steps, prec, tile, seed, flags=0, **kw):
    phi, psi, src = wall_droplet(nx, ny, seed)
    par = dict(ACTIVE, **kw)
    sim = lbd.Sim(nx, ny, precision=prec, sources=src, flags=lbd.LBD_WALLS | flags, **par)
    sim.set_tile(*tile)
    sim.set_fields(phi, psi)
    sim.step(steps)
    ref = oracle.State(oracle.Params(nx, ny, sources=src, flags=oracle.WALLS | flags, **par),
                       phi, psi).step(steps)
    return sim, ref


@pytest.mark.parametrize("nx,ny,tile", [(128, 64, (118, 64)), (128, 64, (246, 32)),
                                        (161, 70, (118, 32)), (100, 23, (118, 64)),
                                        (40, 8, (118, 32)), (300, 130, (246, 64)),
                                        # tiled kernel: whole and partial last tiles
                                        (128, 64, (32, 8)), (161, 70, (32, 16)),
                                        (100, 23, (64, 8)), (40, 8, (32, 8)),
                                        (64, 9, (32, 8)), (300, 130, (32, 32)),
                                        (70, 13, (64, 16))])
def test_fp64_walls_match_oracle(nx, ny, tile):
    sim, ref = run_both(nx, ny, 300, lbd.LBD_FP64, tile, seed=nx + 7 * ny)
    for g, r in zip(sim.fields(), ref.fields()):
        assert rel(g, r) <= 1e-10
    assert rel(sim.populations(), ref.f) <= 1e-10
    sim.close()


@pytest.mark.parametrize("tile", [(118, 64), (32, 8)])
def test_fp32_walls_match_oracle(tile):
    sim, ref = run_both(256, 96, 600, lbd.LBD_FP32, tile, seed=3)
    g, r = sim.fields(), ref.fields()
    for k in (1, 2, 3, 4):
        assert np.abs(g[k] - r[k]).max() <= 1e-4, k
    sim.close()


def test_stripe_shapes_identical_with_walls():
    outs = []
    for tile in ((118, 16), (118, 32), (118, 64), (118, 128), (246, 32), (246, 64)):
        phi, psi, src = wall_droplet(300, 90, 11)
        sim = lbd.Sim(300, 90, precision=lbd.LBD_FP32, sources=src, flags=lbd.LBD_WALLS, **ACTIVE)
        sim.set_tile(*tile)
        sim.set_fields(phi, psi)
        sim.step(80)
        outs.append((sim.fields(), sim.populations()))
        sim.close()
    for o in outs[1:]:
        for a, b in zip(o[0], outs[0][0]):
            assert np.array_equal(a, b)
        assert np.array_equal(o[1], outs[0][1])


def test_initial_populations_with_walls():
    """set_fields stores f^eq(n, u) in the pull layout with the bounce-back
    convention at the plates: the pre-collision populations read back equal
    the oracle's f^eq at every site."""
    nx, ny = 40, 12
    rng = np.random.default_rng(2)
    phi = 0.3 * rng.normal(size=(ny, nx))
    psi = 0.1 + 0.01 * rng.random((ny, nx))
    rho = 1 + 0.01 * rng.normal(size=(ny, nx))
    ux, uy = 0.02 * rng.normal(size=(ny, nx)), 0.02 * rng.normal(size=(ny, nx))
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP64, flags=lbd.LBD_WALLS)
    sim.set_fields(phi, psi, rho=rho, ux=ux, uy=uy)
    ref = oracle.State(oracle.Params(nx, ny, flags=oracle.WALLS), phi, psi, rho=rho, ux=ux, uy=uy)
    assert np.abs(sim.populations() - ref.f).max() <= 1e-15
    sim.close()


def test_poiseuille_on_gpu():
    """Body-force channel flow at tau = 1/2 + sqrt(3)/4, where halfway
    bounce-back gives the parabola with the plates at -1/2 and ny - 1/2
    exactly (FP64)."""
    nx, ny, F = 16, 24, 1e-6
    tau = 0.5 + np.sqrt(3) / 4
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP64, flags=lbd.LBD_WALLS | lbd.LBD_BODY_FORCE,
                  fx=F, tau=tau, **{k: v for k, v in inputs.PAPER.items() if k != "tau"})
    sim.set_fields(np.zeros((ny, nx)), np.full((ny, nx), 0.1))
    sim.step(12000)
    ux = sim.fields()[1]
    y = np.arange(ny)
    nu = (tau - 0.5) / 3
    parabola = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(ux - parabola[:, None]).max() <= 1e-9 * parabola.max()
    sim.close()


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32], ids=["fp64", "fp32"])
def test_conservation_with_walls_on_gpu(prec):
    nx, ny = 256, 80
    phi, psi, _ = wall_droplet(nx, ny, 5)
    sim = lbd.Sim(nx, ny, precision=prec, flags=lbd.LBD_WALLS, M=0.5, tau=0.8)
    sim.set_fields(phi, psi)
    d0 = sim.diagnostics(nx / 2, 10)
    sim.step(2000)
    d1 = sim.diagnostics(nx / 2, 10)
    tol = 1e-12 if prec == lbd.LBD_FP64 else 1e-5
    for k in ("sum_rho", "sum_phi", "sum_psi"):
        assert abs(d1[k] - d0[k]) <= tol * abs(d0[k]), k
    assert d1["nonfinite"] == 0
    sim.close()


def test_walls_rejected_where_unsupported():
    sim = lbd.Sim(264, 64, precision=lbd.LBD_FP32, flags=lbd.LBD_WALLS)
    with pytest.raises(lbd.LbdError) as e:  # the 16-byte staged stripe kernel has no walls
        sim.set_tile(116, 64)
    assert e.value.code == lbd.LBD_EINVAL
    sim.set_tile(32, 16)
    with pytest.raises(lbd.LbdError) as e:
        sim.adjoint(10, 5, 132.0)
    assert e.value.code == lbd.LBD_EINVAL
    sim.close()
    with pytest.raises(lbd.LbdError) as e:
        lbd.Sim(64, 6, precision=lbd.LBD_FP64, flags=lbd.LBD_WALLS)
    assert e.value.code == lbd.LBD_EINVAL
