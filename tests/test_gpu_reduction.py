"""Accuracy of the FP32 form of the diagnostics reduction (the S8 sums of rho,
phi and psi, the phi >= 0 mass and centre, the psi and B minima; Sec. 2,
Eqs. 1-3 and 9), on the bench's 2048 x 2048 emulsion after 200 steps of
developed flow and on a ragged 1022 x 517 lattice (its last four-site chunk of
each row holds two sites).

Two checks on the same GPU state:

* against the FP64 oracle's diagnostics of that state (each site's value
  widened exactly from FP32), within bounds derived from FP32 rounding of the
  kernel's per-chunk sums;
* against the exact sum (math.fsum) of those per-chunk FP32 sums, formed here
  in numpy FP32 in the kernel's order (nine populations summed per site, then
  the four sites of a chunk pairwise).  The (sum, compensation) float pairs
  merged by TwoSum carry that exact sum to within a few u^2 of the magnitude
  summed (u = 2^-24), so the test allows 1e-12 of it; a combine that drops a
  compensation anywhere errs by about u = 6e-8 of the total and fails.

The psi minimum is exact (an FP32 value widened).  B = B0 + B1 psi is monotone
in psi, so its minimum sits at the extreme psi in any rounding; the GPU may
form it with one FMA where the oracle rounds twice, so it is held to two ulps
of |B0| + |B| (the product B1 psi may be larger than B itself).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    import oracle.build
    oracle.build.build()
    lbd.load()


def emulsion_state():
    w = inputs.emulsion(n=2048, count=64, seed=5)
    sim = lbd.Sim(2048, 2048, precision=lbd.LBD_FP32, sources=w["sources"], **w["params"])
    sim.set_fields(w["phi"], w["psi"])
    return sim, w["params"], w["sources"]


def ragged_state():
    nx, ny = 1022, 517
    d = dict(x=400.3, y=250.6, R=90.0, psi_mean=0.1, noise=0.01, gx=0.005)
    phi, psi = inputs.droplet_fields(nx, ny, [d], seed=4)
    src = [inputs.default_source(d, nx, ny)]
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP32, sources=src, M=0.5, tau=0.8)
    sim.set_fields(phi, psi)
    return sim, dict(M=0.5, tau=0.8), src


def chunks(a):
    """Rows of FP32 values padded with zeros to whole four-site chunks,
    shaped (ny, nx / 4, 4)."""
    ny, nx = a.shape
    pad = (-nx) % 4
    return np.pad(a, ((0, 0), (0, pad))).reshape(ny, (nx + pad) // 4, 4)


def pair4(c):
    return (c[..., 0] + c[..., 1]) + (c[..., 2] + c[..., 3])


def image(k, frac, n):
    """Integer minimum-image displacement of site index k from floor(ref):
    the FP64 rule d = k - frac, wrapped into [-n/2, n/2)."""
    d = k.astype(np.float64) - frac
    return np.where(d >= 0.5 * n, k - n, np.where(d < -0.5 * n, k + n, k))


def chunk_sums(f, phi, psi, refx, refy):
    """The kernel's per-chunk FP32 values, from the pre-collision populations
    f (FP64, exact widenings of w_i + g) and the FP32 fields."""
    ny, nx = phi.shape
    site = np.zeros((ny, nx), np.float32)
    for i in range(9):
        # the stored (pull-layout) value at z is f_i(z + e_i) - w_i, exact in FP32
        g = np.roll(f[i], shift=(-EY[i], -EX[i]), axis=(0, 1)) - W[i]
        site = site + g.astype(np.float32)
    p32, c32 = phi.astype(np.float32), psi.astype(np.float32)
    ix, iy = math.floor(refx), math.floor(refy)
    kx = image(np.arange(nx) - ix, refx - ix, nx)
    ky = image(np.arange(ny) - iy, refy - iy, ny)
    m = np.where(p32 >= 0, p32, np.float32(0))
    mc = chunks(m)
    kxc = chunks(np.broadcast_to(kx, (ny, nx)).astype(np.float32))
    cx = np.zeros(mc.shape[:2], np.float32)
    cw = np.zeros(mc.shape[:2], np.float32)
    for k in range(4):
        cx = fma32(mc[..., k], kxc[..., k], cx)
        cw = cw + mc[..., k]
    cy = (cw.astype(np.float64) * ky[:, None]).astype(np.float32)
    return dict(g=pair4(chunks(site)), phi=pair4(chunks(p32)), psi=pair4(chunks(c32)),
                cx=cx, cy=cy, w=cw), (refx - ix, refy - iy)


def fma32(a, b, c):
    """fmaf(a, b, c) for FP32 arrays a, c and integer-valued b (|b| < 2^24):
    a b is exact in FP64; s = a b + c is rounded there once, its error e is
    recovered by TwoSum, and e decides the one case where rounding s to FP32
    differs from rounding the exact a b + c, an FP32 midpoint."""
    p = a.astype(np.float64) * b
    c = c.astype(np.float64)
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    r = s.astype(np.float32)
    rd = r.astype(np.float64)
    d = s - rd
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(-np.inf))
    tie_up = (d > 0) & (2 * d == up.astype(np.float64) - rd) & (e > 0)
    tie_dn = (d < 0) & (2 * d == dn.astype(np.float64) - rd) & (e < 0)
    return np.where(tie_up, up, np.where(tie_dn, dn, r))


def fsum(a):
    a = np.asarray(a, np.float64).ravel()
    return math.fsum(a), float(np.abs(a).sum())


REFS = {"emulsion": [(1024.0, 1024.0), (3.0, 2047.5), (1500.37, 17.81)],
        "ragged": [(400.3, 250.6), (1021.5, 0.25), (7.75, 516.0)]}


@pytest.mark.parametrize("case", ["emulsion", "ragged"])
def test_fp32_reduction_accuracy(case):
    sim, params, src = emulsion_state() if case == "emulsion" else ragged_state()
    sim.step(200)
    f = sim.populations()
    _, _, _, phi, psi = sim.fields()
    ny, nx = phi.shape
    ref = oracle.State(oracle.Params(nx, ny, sources=src, **params), phi, psi, t=sim.t)
    ref.f[...] = f
    for refx, refy in REFS[case]:
        g = sim.diagnostics(refx, refy)
        r = ref.diagnostics(refx, refy)
        cs, (frx, fry) = chunk_sums(f, phi, psi, refx, refy)
        assert g["nonfinite"] == 0 and r["nonfinite"] == 0
        # the exact sums of the FP32 chunk values
        for key, name, base in (("sum_rho", "g", nx * ny), ("sum_phi", "phi", 0),
                                ("sum_psi", "psi", 0), ("mass_pos", "w", 0)):
            s, mag = fsum(cs[name])
            assert abs(g[key] - (base + s)) <= 1e-12 * mag + 1e-12 * base, (case, key)
        sw, _ = fsum(cs["w"])
        sx, mx = fsum(cs["cx"])
        sy, my = fsum(cs["cy"])
        ex = refx + (sx - frx * sw) / sw
        ey = refy + (sy - fry * sw) / sw
        assert abs(g["cm_x"] - ex) <= 1e-12 * (mx / sw + nx), case
        assert abs(g["cm_y"] - ey) <= 1e-12 * (my / sw + ny), case
        # the FP64 oracle on the same state, within the FP32 chunk rounding:
        # a chunk of k terms errs by at most k u of the magnitudes it sums
        gabs = np.abs(f - np.array(W)[:, None, None]).sum()
        assert abs(g["sum_rho"] - r["sum_rho"]) <= 12 * U * gabs
        assert abs(g["sum_phi"] - r["sum_phi"]) <= 3 * U * np.abs(phi).sum()
        assert abs(g["sum_psi"] - r["sum_psi"]) <= 3 * U * np.abs(psi).sum()
        assert abs(g["mass_pos"] - r["mass_pos"]) <= 4 * U * r["mass_pos"]
        bound = 8 * U * (max(nx, ny) + 1)
        assert abs(g["cm_x"] - r["cm_x"]) <= bound and abs(g["cm_y"] - r["cm_y"]) <= bound
        assert g["min_psi"] == r["min_psi"] == psi.min()
        # B0 + B1 psi: the GPU may fuse it into one FMA where the oracle rounds
        # the product too, an ulp of |B1 psi| <= |B0| + |B|
        b0 = ref.p["B0"]
        assert abs(g["min_B"] - r["min_B"]) <= 2 * np.spacing(abs(b0) + abs(r["min_B"]))
    sim.close()
