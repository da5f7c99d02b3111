"""Pins of the 3D (D3Q19) oracle.

* Reduction to 2D: with fields independent of z and no z velocity, the D3Q19
  weights summed over e_z are the D2Q9 weights, so the 3D step must reproduce
  the (separately pinned) 2D oracle: phi, psi, rho, u after 60 steps, with
  source, sink, body force or frozen velocity.
* D3Q19 moments: sum f_eq = n, sum f_eq e = n u, sum f_eq e e = n/3 I + n u u;
  Guo term: sum F_i = 0, sum F_i e = (1 - 1/(2 tau)) F,
  sum F_i e e = (1 - 1/(2 tau)) (u F + F u).
* Stencils along an axis: plane waves give the 3-point results, lap = 2 (cos k - 1)
  and d/dx = sin k, on every axis.
* Conservation of n, phi, psi on a random 3D state.
* Symmetry: exchanging the x and y axes of the state exchanges the result.
"""
import numpy as np
import pytest

import oracle
from oracle import oracle3 as O3


@pytest.fixture(scope="module", autouse=True)
def built():
    import oracle.build
    oracle.build.build()


def random_2d(nx, ny, seed):
    rng = np.random.default_rng(seed)
    phi = 0.6 * np.tanh(2 * rng.normal(size=(ny, nx)))
    psi = 0.1 + 0.005 * rng.random((ny, nx))
    ux, uy = 0.01 * rng.normal(size=(ny, nx)), 0.01 * rng.normal(size=(ny, nx))
    rho = 1 + 0.01 * rng.normal(size=(ny, nx))
    return phi, psi, rho, ux, uy


@pytest.mark.parametrize("nz,flags,kw", [
    (1, 0, dict(gamma=1e-3, c0=0.09, A0=1e-5, A_max=1e-4, t_on=10)),
    (4, 0, dict(M=0.5, tau=0.8)),
    (3, 2, dict(fx=2e-5, fy=-1e-5)),
    (2, 1, dict(ux0=0.03, uy0=-0.02)),
])
def test_reduces_to_2d(nz, flags, kw):
    nx, ny = 24, 20
    phi, psi, rho, ux, uy = random_2d(nx, ny, 7 + nz)
    kw = dict(dict(B1=-0.02), **kw)
    src2 = [(8.0, 9.0, 3.0)] if nz == 1 else []
    src3 = [(8.0, 9.0, 0.0, 3.0)] if nz == 1 else []
    p2 = {k: v for k, v in kw.items() if k not in ("fx", "fy", "ux0", "uy0")}
    extra = {k: kw[k] for k in ("fx", "fy", "ux0", "uy0") if k in kw}
    s2 = oracle.State(oracle.Params(nx, ny, sources=src2, flags=flags, **extra, **p2),
                      phi, psi, rho=rho, ux=ux, uy=uy).step(60)
    rep = lambda a: np.repeat(a[None], nz, axis=0)
    u3 = np.stack([rep(ux), rep(uy), np.zeros((nz, ny, nx))])
    s3 = O3.State3(O3.Params3(nx, ny, nz, sources=src3, flags=flags, **extra, **p2),
                   rep(phi), rep(psi), rho=rep(rho), u=u3).step(60)
    r2, ux2, uy2, ph2, ps2 = s2.fields()
    r3, u3, ph3, ps3 = s3.fields()
    for z in range(nz):
        for a, b in ((ph3[z], ph2), (ps3[z], ps2), (r3[z], r2), (u3[0, z], ux2), (u3[1, z], uy2)):
            assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-2)
    assert np.abs(u3[2]).max() <= 1e-16


def test_d3q19_moments():
    E = np.array([O3.EX, O3.EY, O3.EZ], dtype=float)
    n, u = 1.03, np.array([0.02, -0.03, 0.015])
    feq = O3.equilibrium(n, *u)
    assert feq.sum() == pytest.approx(n, rel=1e-15)
    assert np.allclose(E @ feq, n * u, rtol=0, atol=1e-16)
    assert np.allclose((E * feq) @ E.T, n / 3 * np.eye(3) + n * np.outer(u, u), rtol=0, atol=1e-15)
    tau, F = 0.8, np.array([1e-3, 2e-3, -5e-4])
    Fi = O3.guo(tau, u, F)
    g = 1 - 0.5 / tau
    assert abs(Fi.sum()) <= 1e-18
    assert np.allclose(E @ Fi, g * F, rtol=0, atol=1e-18)
    assert np.allclose((E * Fi) @ E.T, g * (np.outer(u, F) + np.outer(F, u)), rtol=0, atol=1e-18)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_axis_plane_waves(axis):
    L = [16, 12, 10]
    p = O3.Params3(L[0], L[1], L[2])
    m = 3
    k = 2 * np.pi * m / L[axis]
    z, y, x = np.mgrid[0:L[2], 0:L[1], 0:L[0]].astype(float)
    coord = [x, y, z][axis]
    g = np.cos(k * coord)
    assert np.abs(O3.lap(p, g) - 2 * (np.cos(k) - 1) * g).max() <= 1e-14
    grads = O3.grad(p, g)
    assert np.abs(grads[axis] + np.sin(k) * np.sin(k * coord)).max() <= 1e-14
    for a in range(3):
        if a != axis:
            assert np.abs(grads[a]).max() <= 1e-15


def random_3d(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    phi = 0.6 * np.tanh(2 * rng.normal(size=(nz, ny, nx)))
    psi = 0.1 + 0.005 * rng.random((nz, ny, nx))
    u = 0.01 * rng.normal(size=(3, nz, ny, nx))
    return phi, psi, u


def test_conservation_3d():
    nx, ny, nz = 10, 9, 8
    phi, psi, u = random_3d(nx, ny, nz, 3)
    s = O3.State3(O3.Params3(nx, ny, nz, B1=-0.02, M=0.5, tau=0.7), phi, psi, u=u)
    n0, p0, c0 = s.f.sum(), s.phi.sum(), s.psi.sum()
    s.step(40)
    assert abs(s.f.sum() - n0) <= 1e-12 * n0
    assert abs(s.phi.sum() - p0) <= 1e-12 * np.abs(phi).sum()
    assert abs(s.psi.sum() - c0) <= 1e-12 * c0


def test_axis_exchange_symmetry():
    nx = ny = 10
    nz = 7
    phi, psi, u = random_3d(nx, ny, nz, 5)
    kw = dict(B1=-0.02, M=0.5, tau=0.9)
    a = O3.State3(O3.Params3(nx, ny, nz, **kw), phi, psi, u=u).step(20)
    sw = lambda f: np.ascontiguousarray(np.swapaxes(f, -1, -2))
    ub = np.stack([sw(u[1]), sw(u[0]), sw(u[2])])
    b = O3.State3(O3.Params3(nx, ny, nz, **kw), sw(phi), sw(psi), u=ub).step(20)
    ra, ua, pa, qa = a.fields()
    rb, ub2, pb, qb = b.fields()
    assert np.abs(sw(pa) - pb).max() <= 1e-13
    assert np.abs(sw(qa) - qb).max() <= 1e-13
    assert np.abs(sw(ua[0]) - ub2[1]).max() <= 1e-13
    assert np.abs(sw(ua[2]) - ub2[2]).max() <= 1e-13
