"""Pins of the oracle's per-droplet tracking and squirmer fit (Section 4,
Eq. 21), against closed forms: exact centres of symmetric disks (one across
the periodic boundary), a uniform flow returned as the droplet velocity with no
squirmer modes, a rigid rotation with no squirmer modes, and a synthetic
squirmer field whose b1, b2 the fit returns (within the error of the linear
interpolation along the links, O(1/R^2))."""
import numpy as np
import pytest

from oracle import droplets as D


def disk(nx, ny, cx, cy, R, xi=2.0, wrap_y=True):
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    dx = xx - cx
    dx -= nx * np.round(dx / nx)
    dy = yy - cy
    if wrap_y:
        dy -= ny * np.round(dy / ny)
    r = np.hypot(dx, dy)
    return np.tanh((R - r) / xi), dx, dy, r


def two_disks(nx=128, ny=96):
    a, *_ = disk(nx, ny, 20.0, 30.5, 12.0)
    b, *_ = disk(nx, ny, 0.5, 60.0, 15.0)
    return np.maximum(a, b)


def test_centres_of_symmetric_disks():
    nx, ny = 128, 96
    phi = two_disks(nx, ny)
    z = np.zeros_like(phi)
    out = D.droplets(phi, z, z, [(23.0, 27.0), (125.0, 57.0)])
    assert out[0]["x"] == pytest.approx(20.0, abs=1e-12)
    assert out[0]["y"] == pytest.approx(30.5, abs=1e-12)
    assert out[1]["x"] == pytest.approx(0.5, abs=1e-12)
    assert out[1]["y"] == pytest.approx(60.0, abs=1e-12)
    # every phi >= 0 site is counted once
    assert out[0]["sites"] + out[1]["sites"] == int((phi >= 0).sum())
    assert out[0]["mass"] + out[1]["mass"] == pytest.approx(phi[phi >= 0].sum(), rel=1e-14)


def test_uniform_flow():
    nx, ny = 128, 96
    phi = two_disks(nx, ny)
    ux, uy = np.full_like(phi, 0.01), np.full_like(phi, -0.02)
    ds = D.droplets(phi, ux, uy, [(20.0, 30.5), (0.5, 60.0)])
    for d in ds:
        assert d["ux"] == pytest.approx(0.01, rel=1e-13)
        assert d["uy"] == pytest.approx(-0.02, rel=1e-13)
    for f in D.squirmer(phi, ux, uy, ds):
        assert abs(f["b1"]) < 1e-15 and abs(f["b2"]) < 1e-15 and f["points"] > 40


def test_rigid_rotation_has_no_squirmer_modes():
    nx, ny = 96, 96
    phi, dx, dy, r = disk(nx, ny, 48.0, 48.0, 20.0)
    om, U = 1e-3, (0.004, 0.001)
    ux, uy = U[0] - om * dy, U[1] + om * dx
    d = D.droplets(phi, ux, uy, [(48.0, 48.0)])[0]
    assert d["ux"] == pytest.approx(U[0], abs=1e-15)
    assert d["uy"] == pytest.approx(U[1], abs=1e-15)
    f = D.squirmer(phi, ux, uy, [d])[0]
    assert abs(f["b1"]) < 1e-14 and abs(f["b2"]) < 1e-14


@pytest.mark.parametrize("alpha,b1,b2", [(0.0, 2e-3, -1e-3), (0.7, 1e-3, 5e-4), (2.5, -1e-3, 2e-3)])
def test_synthetic_squirmer(alpha, b1, b2):
    nx, ny = 160, 160
    phi, dx, dy, r = disk(nx, ny, 80.0, 80.0, 40.0)
    e = np.array([np.cos(alpha), np.sin(alpha)])
    ep = np.array([-e[1], e[0]])
    U = 3e-3 * e
    rs = np.where(r > 0, r, 1.0)
    c = (dx * e[0] + dy * e[1]) / rs
    s = (dx * ep[0] + dy * ep[1]) / rs
    ut = b1 * s + 0.5 * b2 * (2 * s * c)
    eth_x, eth_y = -s * e[0] + c * ep[0], -s * e[1] + c * ep[1]
    ux, uy = U[0] + ut * eth_x, U[1] + ut * eth_y
    drop = dict(x=80.0, y=80.0, ux=U[0], uy=U[1])
    f = D.squirmer(phi, ux, uy, [drop])[0]
    tol = 5e-3 * max(abs(b1), abs(b2))
    assert f["b1"] == pytest.approx(b1, abs=tol)
    assert f["b2"] == pytest.approx(b2, abs=tol)
    assert f["points"] > 200


def test_plates_stop_the_wrap_in_y():
    nx, ny = 80, 40
    phi, *_ = disk(nx, ny, 40.0, 1.0, 10.0)
    z = np.zeros_like(phi)
    periodic = D.droplets(phi, z, z, [(40.0, 1.0)])[0]
    walled = D.droplets(phi, z, z, [(40.0, 1.0)], walls=True)[0]
    assert periodic["y"] == pytest.approx(1.0, abs=1e-12)
    assert walled["y"] > 5.0  # the rows near y = ny - 1 are far from the droplet
