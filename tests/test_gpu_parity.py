"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

Tolerances: FP64 GPU, max relative field error <= 1e-10 per field
(||X_gpu - X_orc||_inf / ||X_orc||_inf) after up to 2000 steps; FP32 GPU
(shifted populations), phi, psi and u within 1e-4 absolute and the droplet
centroid within 0.02 lattice units over the run.
"""
import numpy as np
import pytest

import oracle
from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu

NAMES = ["rho", "ux", "uy", "phi", "psi"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    import oracle.build
    oracle.build.build()
    lbd.load()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def run_both(nx, ny, phi, psi, steps, precision=lbd.LBD_FP64, sources=(), tile=None,
             rho=None, ux=None, uy=None, flags=0, **kw):
    sim = lbd.Sim(nx, ny, precision=precision, sources=sources, flags=flags, **kw)
    if tile:
        sim.set_tile(*tile)
    sim.set_fields(phi, psi, rho=rho, ux=ux, uy=uy)
    sim.step(steps)
    ref = oracle.State(oracle.Params(nx, ny, sources=sources, flags=flags, **kw), phi, psi,
                       rho=rho, ux=ux, uy=uy).step(steps)
    return sim, ref


ACTIVE = dict(M=0.5, tau=0.8, gamma=1.5e-3, c0=0.09, A0=1e-7, A_max=1e-4, t_on=300)


def droplet(nx, ny, seed=1, R=None):
    d = dict(x=nx / 2 - 0.3, y=ny / 2 + 0.4, R=R or min(nx, ny) / 4, psi_mean=0.1, noise=0.01,
             gx=0.005)
    phi, psi = inputs.droplet_fields(nx, ny, [d], seed=seed)
    return d, phi, psi


KERNELS = [(32, 16), (118, 64), (246, 32)]   # tiled, stripe (1 column per thread)


@pytest.mark.parametrize("tile", KERNELS, ids=lambda t: "%dx%d" % t)
def test_fp64_single_droplet_1000_steps(tile):
    """128^2 droplet with source, sink and schedule on: FP64 GPU matches the
    oracle to 1e-10 relative per field after 1000 steps (tiled kernel and
    stripe-marching kernel)."""
    n = 128
    d, phi, psi = droplet(n, n, seed=1, R=20)
    src = [inputs.default_source(d, n, n)]
    sim, ref = run_both(n, n, phi, psi, 1000, sources=src, tile=tile, **ACTIVE)
    for g, r, name in zip(sim.fields(), ref.fields(), NAMES):
        assert rel_err(g, r) <= 1e-10, name
    f = sim.populations()
    assert rel_err(f, ref.f) <= 1e-10


def test_fp64_config1_2000_steps():
    """The 128^2 single-droplet workload as shipped (passive 1000 steps, then the
    sink and the source ramp), 2000 steps."""
    w = inputs.single_droplet()
    sim, ref = run_both(w["nx"], w["ny"], w["phi"], w["psi"], 2000, sources=w["sources"],
                        **w["params"])
    for g, r, name in zip(sim.fields(), ref.fields(), NAMES):
        assert rel_err(g, r) <= 1e-10, name


@pytest.mark.parametrize("tile", KERNELS, ids=lambda t: "%dx%d" % t)
@pytest.mark.parametrize("nx,ny", [(100, 37), (37, 100), (8, 8), (5, 4), (161, 23), (300, 130)])
def test_fp64_ragged_and_small_grids(nx, ny, tile):
    """Grids that span several tiles or stripes with a ragged tail, and grids
    smaller than one tile (the halo wraps several times)."""
    d, phi, psi = droplet(nx, ny, seed=nx * 1000 + ny, R=max(2.0, min(nx, ny) / 4))
    src = [(nx / 3, ny / 2, max(1.0, min(nx, ny) / 8))]
    sim, ref = run_both(nx, ny, phi, psi, 150, sources=src, tile=tile,
                        **dict(ACTIVE, t_on=20, A0=1e-6))
    for g, r, name in zip(sim.fields(), ref.fields(), NAMES):
        assert rel_err(g, r) <= 1e-10, name


def family(t):
    if t[0] <= 64:
        return "tiled"
    return "vstripe" if t[0] == 116 else "stripe"


def test_tiles_give_identical_results():
    """Each site's arithmetic does not depend on the launch shape: all shapes of
    one kernel produce bit-identical states, and the kernels (different
    operation order) agree to rounding."""
    nx, ny = 300, 70
    d, phi, psi = droplet(nx, ny, seed=5)
    src = [inputs.default_source(d, nx, ny)]
    outs = []
    for t in lbd.tiles():
        for prec in (lbd.LBD_FP64, lbd.LBD_FP32):
            if family(t) == "vstripe" and prec == lbd.LBD_FP64:
                continue
            sim = lbd.Sim(nx, ny, precision=prec, sources=src, **dict(ACTIVE, t_on=10, A0=1e-6))
            sim.set_tile(*t)
            sim.set_fields(phi, psi)
            sim.step(60)
            outs.append((prec, t, sim.fields(), sim.populations()))
    for prec in (lbd.LBD_FP64, lbd.LBD_FP32):
        fams = ["tiled", "stripe"] + (["vstripe"] if prec == lbd.LBD_FP32 else [])
        for fam in fams:
            base = [o for o in outs if o[0] == prec and family(o[1]) == fam]
            assert base, fam
            for o in base[1:]:
                for a, b in zip(o[2], base[0][2]):
                    assert np.array_equal(a, b), (prec, o[1])
                assert np.array_equal(o[3], base[0][3])
        tiled = [o for o in outs if o[0] == prec and family(o[1]) == "tiled"][0]
        tol = 1e-12 if prec == lbd.LBD_FP64 else 1e-5
        for fam in fams[1:]:
            other = [o for o in outs if o[0] == prec and family(o[1]) == fam][0]
            for a, b in zip(tiled[2], other[2]):
                assert np.abs(a - b).max() <= tol * max(np.abs(a).max(), 1e-3), fam


@pytest.mark.parametrize("tile", KERNELS, ids=lambda t: "%dx%d" % t)
def test_fp32_shifted_populations_tolerance(tile):
    """FP32 form over the 2000-step single-droplet workload: phi, psi, u within
    1e-4 absolute of the FP64 oracle, and the centroid within 0.02."""
    w = inputs.single_droplet()
    n = w["nx"]
    sim = lbd.Sim(n, n, precision=lbd.LBD_FP32, sources=w["sources"], **w["params"])
    sim.set_tile(*tile)
    sim.set_fields(w["phi"], w["psi"])
    ref = oracle.State(oracle.Params(n, n, sources=w["sources"], **w["params"]), w["phi"], w["psi"])
    for _ in range(4):
        sim.step(500)
        ref.step(500)
        g, r = sim.fields(), ref.fields()
        for k in (1, 2, 3, 4):
            assert np.abs(g[k] - r[k]).max() <= 1e-4, NAMES[k]
        dg, dr = sim.diagnostics(64, 64), ref.diagnostics(64, 64)
        assert abs(dg["cm_x"] - dr["cm_x"]) <= 0.02 and abs(dg["cm_y"] - dr["cm_y"]) <= 0.02


@pytest.mark.parametrize("tile", [(116, 64), (116, 32), (118, 64)], ids=lambda t: "%dx%d" % t)
def test_fp32_two_droplets_512x256(tile):
    """FP32 on the 512x256 two-droplet workload: phi, psi, u within 1e-4 of the
    FP64 oracle after 600 steps with source and sink on, and the centroid
    within 0.02."""
    w = inputs.two_droplets(sep=80.0, offset=20.0)
    nx, ny = w["nx"], w["ny"]
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP32, sources=w["sources"], **w["params"])
    sim.set_tile(*tile)
    sim.set_fields(w["phi"], w["psi"])
    ref = oracle.State(oracle.Params(nx, ny, sources=w["sources"], **w["params"]), w["phi"], w["psi"])
    for _ in range(2):
        sim.step(300)
        ref.step(300)
        g, r = sim.fields(), ref.fields()
        for k in (1, 2, 3, 4):
            assert np.abs(g[k] - r[k]).max() <= 1e-4, NAMES[k]
        for d in w["droplets"]:
            dg, dr = sim.diagnostics(d["x"], d["y"]), ref.diagnostics(d["x"], d["y"])
            assert abs(dg["cm_x"] - dr["cm_x"]) <= 0.02 and abs(dg["cm_y"] - dr["cm_y"]) <= 0.02


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
def test_diagnostics_match_oracle(prec):
    nx, ny = 96, 80
    d, phi, psi = droplet(nx, ny, seed=9)
    src = [inputs.default_source(d, nx, ny)]
    sim, ref = run_both(nx, ny, phi, psi, 200, precision=prec, sources=src,
                        **dict(ACTIVE, t_on=0, A0=1e-6))
    # the moving reference point exercises the minimum image
    for refx, refy in [(d["x"], d["y"]), (3.0, 77.5), (90.0, 2.0)]:
        g, r = sim.diagnostics(refx, refy), ref.diagnostics(refx, refy)
        tol = 1e-12 if prec == lbd.LBD_FP64 else 2e-4
        for k in ("sum_rho", "sum_phi", "sum_psi", "mass_pos"):
            assert abs(g[k] - r[k]) <= tol * max(abs(r[k]), 1.0) * (1 if prec == 0 else 10), k
        ctol = 1e-10 if prec == lbd.LBD_FP64 else 0.02
        assert abs(g["cm_x"] - r["cm_x"]) <= ctol and abs(g["cm_y"] - r["cm_y"]) <= ctol
        assert g["min_B"] == pytest.approx(r["min_B"], rel=1e-9 if prec == 0 else 1e-3)
        assert g["min_psi"] == pytest.approx(r["min_psi"], rel=1e-12 if prec == 0 else 1e-5)
        assert g["nonfinite"] == 0


def test_conservation_on_gpu():
    """FP64: totals of rho, phi (and psi with activity off) drift only by
    rounding; FP32: drift stated and bounded."""
    nx, ny = 128, 96
    d, phi, psi = droplet(nx, ny, seed=3)
    for prec, tol in ((lbd.LBD_FP64, 1e-13), (lbd.LBD_FP32, 1e-6)):
        sim = lbd.Sim(nx, ny, precision=prec, M=0.5, tau=0.8)
        sim.set_fields(phi, psi)
        d0 = sim.diagnostics(64, 48)
        sim.step(1000)
        d1 = sim.diagnostics(64, 48)
        for k in ("sum_rho", "sum_phi", "sum_psi"):
            assert abs(d1[k] - d0[k]) <= tol * abs(d0[k]) + tol, (prec, k)


def test_body_force_and_frozen_velocity_flags():
    nx, ny = 40, 36
    F = (1e-5, -2e-5)
    sim = lbd.Sim(nx, ny, flags=lbd.LBD_BODY_FORCE, fx=F[0], fy=F[1])
    sim.set_fields(np.full((ny, nx), 0.9), np.full((ny, nx), 0.1))
    sim.step(25)
    f = sim.populations()
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    jx = np.einsum("iyx,i->", f, ex)
    jy = np.einsum("iyx,i->", f, ey)
    assert jx == pytest.approx(F[0] * 25 * nx * ny, rel=1e-11)
    assert jy == pytest.approx(F[1] * 25 * nx * ny, rel=1e-11)
    d, phi, psi = droplet(nx, ny, seed=2)
    kw = dict(ux0=0.05, uy0=-0.03, M=0.3)
    sim, ref = run_both(nx, ny, phi, psi, 100, flags=lbd.LBD_FROZEN_U, **kw)
    for g, r, name in zip(sim.fields(), ref.fields(), NAMES):
        assert rel_err(g, r) <= 1e-10, name


def test_initial_velocity_and_density():
    """Non-uniform initial rho and u set through the ABI (equilibrium populations)."""
    nx, ny = 64, 48
    d, phi, psi = droplet(nx, ny, seed=4)
    rng = np.random.default_rng(0)
    rho = 1 + 0.01 * rng.standard_normal((ny, nx))
    ux = 0.01 * rng.standard_normal((ny, nx))
    uy = 0.01 * rng.standard_normal((ny, nx))
    sim, ref = run_both(nx, ny, phi, psi, 100, rho=rho, ux=ux, uy=uy)
    for g, r, name in zip(sim.fields(), ref.fields(), NAMES):
        assert rel_err(g, r) <= 1e-10, name


def test_error_paths():
    nx, ny = 16, 16
    sim = lbd.Sim(nx, ny)
    phi = np.zeros((ny, nx))
    psi = np.full((ny, nx), 0.1)
    bad = phi.copy()
    bad[3, 4] = np.nan
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields(bad, psi)
    assert e.value.code == lbd.LBD_ENONFINITE
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields(phi, np.full((ny, nx), 0.2))  # B = 0.006 - 0.05*0.2 < 0
    assert e.value.code == lbd.LBD_EUNSTABLE
    # the first bad site in index order, and the first failing test of that site
    two = psi.copy()
    two[2, 7] = -1.0   # site 39: psi <= 0
    bad2 = phi.copy()
    bad2[5, 1] = np.inf  # site 81
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields(bad2, two)
    assert e.value.code == lbd.LBD_EUNSTABLE and "site 39" in str(e.value)
    bad3 = phi.copy()
    bad3[2, 7] = np.nan  # site 39 is both non-finite (phi) and unstable (psi)
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields(bad3, two)
    assert e.value.code == lbd.LBD_ENONFINITE and "site 39" in str(e.value)
    rho = np.ones((ny, nx))
    rho[0, 3] = 0.0
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields(phi, psi, rho=rho)
    assert e.value.code == lbd.LBD_EINVAL and "site 3" in str(e.value)
    # a rejected upload leaves the state as it was
    good = np.tanh(np.linspace(-2, 2, nx))[None, :].repeat(ny, 0)
    sim.set_fields(good, psi)
    before = sim.fields()
    with pytest.raises(lbd.LbdError):
        sim.set_fields(bad, psi)
    for a, b in zip(sim.fields(), before):
        assert np.array_equal(a, b)
    with pytest.raises(lbd.LbdError) as e:
        sim.set_tile(48, 48)
    assert e.value.code == lbd.LBD_EINVAL
    with pytest.raises(lbd.LbdError):
        sim.diagnostics(-1.0, 3.0)
    sim.set_fields(phi, psi)
    sim.step(3)
    assert sim.t == 3


@pytest.mark.parametrize("flags", [0, lbd.LBD_WALLS], ids=["periodic", "plates"])
@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
def test_rest_state_upload_equals_explicit_rest(prec, flags):
    """set_fields without rho and u builds the rest state directly (g = 0); it is
    bit-identical to uploading rho = 1, u = 0 explicitly (the equilibrium
    formula), before and after steps."""
    nx, ny = 60, 44
    d, phi, psi = droplet(nx, ny, seed=12)
    sims = []
    for explicit in (False, True):
        sim = lbd.Sim(nx, ny, precision=prec, flags=flags, **dict(ACTIVE, t_on=0))
        if explicit:
            sim.set_fields(phi, psi, rho=np.ones((ny, nx)), ux=np.zeros((ny, nx)),
                           uy=np.zeros((ny, nx)))
        else:
            sim.set_fields(phi, psi)
        sims.append(sim)
    assert np.array_equal(sims[0].populations(), sims[1].populations())
    for s in sims:
        s.step(30)
    for a, b in zip(sims[0].fields(), sims[1].fields()):
        assert np.array_equal(a, b)
    assert np.array_equal(sims[0].populations(), sims[1].populations())


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
def test_float_upload_and_readback(prec):
    """lbd_set_fields_f32 of float values equals lbd_set_fields of the same values
    held as doubles (the widening is exact), bit for bit, with and without rho
    and u; lbd_get_fields_f32 returns lbd_get_fields rounded to float."""
    nx, ny = 76, 50
    d, phi, psi = droplet(nx, ny, seed=21)
    rng = np.random.default_rng(5)
    f32 = lambda a: np.asarray(a, dtype=np.float32)
    phi32, psi32 = f32(phi), f32(psi)
    rho32 = f32(1 + 0.01 * rng.standard_normal((ny, nx)))
    u32 = [f32(0.01 * rng.standard_normal((ny, nx))) for _ in range(2)]
    for with_u in (False, True):
        sims = []
        for use_f32 in (False, True):
            sim = lbd.Sim(nx, ny, precision=prec, **dict(ACTIVE, t_on=0))
            kw = dict(rho=rho32, ux=u32[0], uy=u32[1]) if with_u else {}
            if use_f32:
                sim.set_fields_f32(phi32, psi32, **kw)
            else:
                sim.set_fields(phi32.astype(np.float64), psi32.astype(np.float64),
                               **{k: v.astype(np.float64) for k, v in kw.items()})
            sims.append(sim)
        assert np.array_equal(sims[0].populations(), sims[1].populations())
        for s in sims:
            s.step(25)
        assert np.array_equal(sims[0].populations(), sims[1].populations())
        got = sims[1].fields_f32()
        for a, b in zip(got, sims[1].fields()):
            assert a.dtype == np.float32
            assert np.array_equal(a, b.astype(np.float32))
        if prec == lbd.LBD_FP32:
            # phi and psi are stored in float: the readback is exact
            assert np.array_equal(got[3].astype(np.float64), sims[1].fields()[3])


def test_float_io_rejects_bad_input():
    nx, ny = 40, 24
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP32)
    d, phi, psi = droplet(nx, ny)
    sim.set_fields_f32(phi, psi)
    before = sim.fields()
    bad = np.asarray(phi, dtype=np.float32).copy()
    bad[3, 5] = np.nan
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields_f32(bad, psi)
    assert e.value.code == lbd.LBD_ENONFINITE
    for a, b in zip(sim.fields(), before):
        assert np.array_equal(a, b)
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields_f32(phi, psi, rho=-np.ones((ny, nx), dtype=np.float32))
    assert e.value.code == lbd.LBD_EINVAL
    r = sim.fields_f32()
    assert np.array_equal(r[3], before[3].astype(np.float32))


def test_float_io_fast_paths_fp32():
    """FP32 context: a float rest-state upload lands in the state only when every
    site is valid (psi <= 0 -> LBD_EUNSTABLE, state unchanged); the float
    read-back fills exactly the arrays asked for (NULL skips a field)."""
    import ctypes
    nx, ny = 52, 36
    d, phi, psi = droplet(nx, ny, seed=3)
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP32, **dict(ACTIVE, t_on=0))
    sim.set_fields_f32(phi, psi)
    sim.step(7)
    before, pops = sim.fields(), sim.populations()
    bad = np.asarray(psi, dtype=np.float32).copy()
    bad[ny - 1, nx - 1] = -0.5
    with pytest.raises(lbd.LbdError) as e:
        sim.set_fields_f32(phi, bad)
    assert e.value.code == lbd.LBD_EUNSTABLE
    for a, b in zip(sim.fields(), before):
        assert np.array_equal(a, b)
    assert np.array_equal(sim.populations(), pops)
    fp = ctypes.POINTER(ctypes.c_float)
    full = sim.fields_f32()
    outs = [np.full((ny, nx), 7.0, dtype=np.float32) for _ in range(5)]
    ask = [False, True, False, False, True]
    ptrs = [o.ctypes.data_as(fp) if a else None for o, a in zip(outs, ask)]
    assert lbd.load().lbd_get_fields_f32(sim._h, *ptrs) == 0
    for o, f, a in zip(outs, full, ask):
        assert np.array_equal(o, f) if a else np.all(o == 7.0)
