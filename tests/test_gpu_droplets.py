"""GPU per-droplet tracking and squirmer fit (lbd_droplets, lbd_squirmer)
against the numpy oracle of Section 4 / Eq. (21) on the same fields.

* Synthetic fields (thermodynamic force switched off, so the evaluated velocity
  is the one uploaded): the GPU and the oracle agree to rounding, and the fit
  returns the b1, b2 of a synthetic squirmer within the interpolation error.
* Evolved states (FP64, periodic and between plates): centres, masses and
  velocities within 1e-10, site and point counts exact, b1 and b2 within 1e-8
  relative of the oracle applied to the oracle's own fields.
"""
import numpy as np
import pytest

import oracle
from oracle import droplets as D
from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu

NOFORCE = dict(a=0.0, b=0.0, B0=1e-30, B1=0.0, tau=0.8, M=0.1, D=0.1)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    import oracle.build
    oracle.build.build()
    lbd.load()


def synthetic(nx, ny, cx, cy, R, alpha, b1, b2, U=3e-3, xi=2.0):
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    dx = xx - cx
    dx -= nx * np.round(dx / nx)
    dy = yy - cy
    dy -= ny * np.round(dy / ny)
    r = np.hypot(dx, dy)
    phi = np.tanh((R - r) / xi)
    e = np.array([np.cos(alpha), np.sin(alpha)])
    ep = np.array([-e[1], e[0]])
    rs = np.where(r > 0, r, 1.0)
    c, s = (dx * e[0] + dy * e[1]) / rs, (dx * ep[0] + dy * ep[1]) / rs
    ut = b1 * s + b2 * s * c
    ux = U * e[0] + ut * (-s * e[0] + c * ep[0])
    uy = U * e[1] + ut * (-s * e[1] + c * ep[1])
    return phi, ux, uy


def test_synthetic_squirmer_on_gpu():
    nx, ny, b1, b2 = 160, 128, 2e-3, -1.5e-3
    phi, ux, uy = synthetic(nx, ny, 70.5, 64.0, 36.0, 0.4, b1, b2)
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP64, **NOFORCE)
    sim.set_fields(phi, np.full((ny, nx), 0.1), ux=ux, uy=uy)
    g = sim.fields()
    assert np.abs(g[1] - ux).max() <= 1e-15 and np.abs(g[2] - uy).max() <= 1e-15
    dg = sim.droplets([(75.0, 60.0)])
    do = D.droplets(phi, ux, uy, [(75.0, 60.0)])
    for k in ("x", "y", "ux", "uy"):
        assert dg[0][k] == pytest.approx(do[0][k], abs=1e-12), k
    assert dg[0]["sites"] == do[0]["sites"]
    assert dg[0]["mass"] == pytest.approx(do[0]["mass"], rel=1e-13)
    # the fit in the frame the synthetic field was built in
    drop = dict(x=70.5, y=64.0, ux=3e-3 * np.cos(0.4), uy=3e-3 * np.sin(0.4))
    fg = sim.squirmer([drop])[0]
    fo = D.squirmer(phi, ux, uy, [drop])[0]
    assert fg["points"] == fo["points"] > 200
    assert fg["b1"] == pytest.approx(fo["b1"], rel=1e-9)
    assert fg["b2"] == pytest.approx(fo["b2"], rel=1e-9)
    assert fg["b1"] == pytest.approx(b1, rel=5e-3)
    assert fg["b2"] == pytest.approx(b2, rel=5e-3)
    sim.close()


@pytest.mark.parametrize("walls", [False, True], ids=["periodic", "plates"])
def test_evolved_droplets_match_oracle(walls):
    w = inputs.two_droplets(nx=256, ny=128, R=20.0, sep=70.0, offset=10.0)
    nx, ny = w["nx"], w["ny"]
    par = dict(w["params"], A0=1e-6, t_on=0)
    flags = lbd.LBD_WALLS if walls else 0
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP64, sources=w["sources"], flags=flags, **par)
    sim.set_fields(w["phi"], w["psi"])
    sim.step(400)
    ref = oracle.State(oracle.Params(nx, ny, sources=w["sources"],
                                     flags=oracle.WALLS if walls else 0, **par),
                       w["phi"], w["psi"]).step(400)
    rho, ux, uy, phi, psi = ref.fields()
    refs = [(d["x"], d["y"]) for d in w["droplets"]]
    dg, do = sim.droplets(refs), D.droplets(phi, ux, uy, refs, walls=walls)
    for a, b in zip(dg, do):
        for k in ("x", "y"):
            assert a[k] == pytest.approx(b[k], abs=1e-10), k
        for k in ("ux", "uy"):
            assert a[k] == pytest.approx(b[k], abs=1e-12), k
        assert a["mass"] == pytest.approx(b["mass"], rel=1e-10)
        assert a["sites"] == b["sites"]
    fg, fo = sim.squirmer(dg), D.squirmer(phi, ux, uy, do, walls=walls)
    for a, b in zip(fg, fo):
        assert a["points"] == b["points"] > 50
        assert a["b1"] == pytest.approx(b["b1"], rel=1e-8)
        assert a["b2"] == pytest.approx(b["b2"], rel=1e-8)
    sim.close()


def test_fp32_droplets_track_fp64():
    w = inputs.two_droplets(nx=256, ny=128, R=20.0, sep=70.0, offset=10.0)
    nx, ny = w["nx"], w["ny"]
    refs = [(d["x"], d["y"]) for d in w["droplets"]]
    out = {}
    for prec in (lbd.LBD_FP64, lbd.LBD_FP32):
        sim = lbd.Sim(nx, ny, precision=prec, sources=w["sources"], **dict(w["params"], t_on=0))
        sim.set_fields(w["phi"], w["psi"])
        sim.step(1000)
        out[prec] = sim.droplets(refs)
        sim.close()
    for a, b in zip(out[lbd.LBD_FP64], out[lbd.LBD_FP32]):
        assert abs(a["x"] - b["x"]) <= 0.02 and abs(a["y"] - b["y"]) <= 0.02


def test_droplet_arguments_checked():
    sim = lbd.Sim(64, 64, precision=lbd.LBD_FP64)
    for refs in ([], [(1.0, 1.0)] * 65, [(64.0, 3.0)], [(3.0, -1.0)]):
        with pytest.raises(lbd.LbdError) as e:
            sim.droplets(refs)
        assert e.value.code == lbd.LBD_EINVAL
    with pytest.raises(lbd.LbdError) as e:
        sim.squirmer([dict(x=float("nan"), y=1.0, ux=0.0, uy=0.0)])
    assert e.value.code == lbd.LBD_EINVAL
    sim.close()
