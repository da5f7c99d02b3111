"""Pins of the oracle's walls (bounce-back plates at y = -1/2 and y = ny - 1/2,
mirrored fields for the finite differences, no advective flux through a plate).

* Poiseuille flow under a body force F between the plates (phi = 0, psi
  uniform, so the thermodynamic force vanishes).  For BGK with halfway
  bounce-back the steady lattice solution is the parabola with the plates at
  y = -1/2 and y = ny - 1/2 plus a uniform slip F (16 L - 3) / (24 nu), with
  L = (tau - 1/2)^2 and nu = (tau - 1/2) / 3; the slip vanishes at
  L = 3/16 (tau = 1/2 + sqrt(3)/4), where the parabola is exact.
* Conservation: total n, phi and psi are kept to rounding with walls.
* Mirror equivalence of the finite-difference part: with a frozen velocity
  along the plates, the walled lattice of height ny evolves exactly as rows
  0..ny-1 of the periodic lattice of height 2 ny holding the fields and their
  mirror image (the plates are the mirror lines of that lattice).
"""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module", autouse=True)
def built():
    import oracle.build
    oracle.build.build()


@pytest.mark.parametrize("tau,steps", [(0.5 + np.sqrt(3) / 4, 12000), (0.8, 16000), (1.0, 12000)])
def test_poiseuille_between_plates(tau, steps):
    nx, ny, F = 4, 24, 1e-6
    P = oracle.Params(nx, ny, flags=oracle.WALLS | oracle.BODY_FORCE, fx=F, tau=tau)
    st = oracle.State(P, np.zeros((ny, nx)), np.full((ny, nx), 0.1))
    st.step(steps)
    rho, ux, uy, _, _ = st.fields()
    nu = (tau - 0.5) / 3
    lam = (tau - 0.5) ** 2
    y = np.arange(ny)
    exact = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y) + F * (16 * lam - 3) / (24 * nu)
    for col in range(nx):
        assert np.abs(ux[:, col] - exact).max() <= 1e-9 * exact.max()
    assert np.abs(uy).max() <= 1e-14
    assert np.abs(rho - 1.0).max() <= 1e-11  # rounding accumulated over the run


def test_plates_exact_at_the_magic_relaxation_time():
    nx, ny, F, tau = 4, 16, 2e-6, 0.5 + np.sqrt(3) / 4
    P = oracle.Params(nx, ny, flags=oracle.WALLS | oracle.BODY_FORCE, fx=F, tau=tau)
    st = oracle.State(P, np.zeros((ny, nx)), np.full((ny, nx), 0.1)).step(9000)
    ux = st.fields()[1][:, 0]
    y = np.arange(ny)
    nu = (tau - 0.5) / 3
    parabola = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(ux - parabola).max() <= 1e-11 * parabola.max()


def random_state(nx, ny, seed):
    rng = np.random.default_rng(seed)
    phi = 0.5 * np.tanh(rng.normal(size=(ny, nx)))
    psi = 0.1 + 0.01 * rng.random((ny, nx))
    ux = 0.02 * rng.normal(size=(ny, nx))
    uy = 0.02 * rng.normal(size=(ny, nx))
    return phi, psi, ux, uy


def test_conservation_with_walls():
    nx, ny = 20, 14
    phi, psi, ux, uy = random_state(nx, ny, 3)
    P = oracle.Params(nx, ny, flags=oracle.WALLS, B1=-0.02, tau=0.7, M=0.5)
    st = oracle.State(P, phi, psi, ux=ux, uy=uy)
    d0 = st.diagnostics(nx / 2, ny / 2)
    st.step(300)
    d1 = st.diagnostics(nx / 2, ny / 2)
    for k in ("sum_rho", "sum_phi", "sum_psi"):
        assert abs(d1[k] - d0[k]) <= 1e-12 * max(abs(d0[k]), 1.0), k
    assert d1["nonfinite"] == 0


def test_finite_differences_mirror_equivalence():
    nx, ny = 12, 10
    phi, psi, _, _ = random_state(nx, ny, 8)
    kw = dict(B1=-0.02, M=0.5, D=0.1, gamma=1e-3, c0=0.09, t_on=0, ux0=0.05, uy0=0.0)
    walled = oracle.State(oracle.Params(nx, ny, flags=oracle.WALLS | oracle.FROZEN_U, **kw), phi, psi)
    dphi, dpsi = np.vstack([phi, phi[::-1]]), np.vstack([psi, psi[::-1]])
    periodic = oracle.State(oracle.Params(nx, 2 * ny, flags=oracle.FROZEN_U, **kw), dphi, dpsi)
    walled.step(40)
    periodic.step(40)
    assert np.abs(walled.phi - periodic.phi[:ny]).max() <= 1e-14
    assert np.abs(walled.psi - periodic.psi[:ny]).max() <= 1e-14
    # and the periodic run kept its mirror symmetry
    assert np.abs(periodic.phi[:ny] - periodic.phi[ny:][::-1]).max() <= 1e-14


def test_walls_break_the_periodic_wrap_in_y():
    """A plate is not periodic: the same initial state evolves differently with
    and without walls."""
    nx, ny = 8, 8
    phi, psi, ux, uy = random_state(nx, ny, 5)
    a = oracle.State(oracle.Params(nx, ny, flags=oracle.WALLS), phi, psi, ux=ux, uy=uy).step(5)
    b = oracle.State(oracle.Params(nx, ny), phi, psi, ux=ux, uy=uy).step(5)
    assert np.abs(a.phi - b.phi).max() > 1e-6
