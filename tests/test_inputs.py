"""The seeded input recipes (no GPU): the properties their docstrings state,
checked on the arrays they build.  The recipes hold none of the method's
arithmetic; these tests keep the workloads the benchmark and the parity tests
start from what they are described to be."""
import math

import numpy as np
import pytest

from paper_1711_10984_gb300 import inputs

PHIEQ = 1.0  # sqrt(-a / b) with a = -b


def min_image_dist(p, q, L):
    d = [inputs._min_image(a - b, L) for a, b in zip(p, q)]
    return math.sqrt(sum(x * x for x in d))


def test_uniform_stream_offsets_and_range():
    a = inputs.uniform01(123, 40)
    assert np.array_equal(inputs.uniform01(123, 15, start=25), a[25:])
    assert a.min() >= 0.0 and a.max() < 1.0
    assert not np.array_equal(a, inputs.uniform01(124, 40))


def test_single_droplet_fields():
    n, R = 96, 20.0
    d = dict(x=40.0, y=50.0, R=R, psi_mean=0.11, noise=0.01, gx=0.004, gy=-0.002)
    phi, psi = inputs.droplet_fields(n, n, [d], seed=7)
    # phi > 0 exactly inside radius R, tanh profile, bounded by phi_eq
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    r = np.hypot(inputs._min_image(xx - 40.0, n), inputs._min_image(yy - 50.0, n))
    assert np.all((phi > 0) == (r < R))
    assert np.abs(phi).max() <= PHIEQ
    # psi: the background outside; mean + noise + ramp inside, within its bounds
    assert np.all(psi[r >= R] == 0.1)
    lo = 0.11 - 0.01 - 0.004 - 0.002
    hi = 0.11 + 0.01 + 0.004 + 0.002
    assert psi[r < R].min() >= lo and psi[r < R].max() <= hi
    # seeded: the same seed gives the same arrays
    phi2, psi2 = inputs.droplet_fields(n, n, [d], seed=7)
    assert np.array_equal(phi, phi2) and np.array_equal(psi, psi2)


def test_droplet_across_the_periodic_edge():
    """A droplet centred near x = 0 is the shifted copy of one centred inside."""
    n = 64
    base = dict(x=32.0, y=30.0, R=12.0)
    edge = dict(x=2.0, y=30.0, R=12.0)
    phi_b, _ = inputs.droplet_fields(n, n, [base])
    phi_e, _ = inputs.droplet_fields(n, n, [edge])
    assert np.array_equal(np.roll(phi_b, -30, axis=1), phi_e)


def test_emulsion_workload():
    """The 2048^2 benchmark emulsion: 64 droplets R = 25 at a minimum-image
    centre distance >= 2R + 4 xi0, one source disk of radius R/4 inside each,
    B(psi) > 0 and psi > 0 everywhere."""
    w = inputs.emulsion(n=2048, count=64, seed=5)
    n, R = 2048, 25.0
    assert len(w["droplets"]) == 64 and len(w["sources"]) == 64
    xi0 = inputs.interface_width(-0.001, 0.006, -0.05, 0.1)
    c = [(d["x"], d["y"]) for d in w["droplets"]]
    dmin = min(min_image_dist(c[i], c[j], n) for i in range(64) for j in range(i))
    assert dmin >= 2 * R + 4 * xi0
    for d, (sx, sy, sr) in zip(w["droplets"], w["sources"]):
        assert sr == R / 4
        assert min_image_dist((sx, sy), (d["x"], d["y"]), n) == pytest.approx(R - sr, abs=1e-9)
    p = w["params"]
    assert w["psi"].min() > 0 and (p["B0"] + p["B1"] * w["psi"]).min() > 0
    assert (w["phi"] > 0).sum() == pytest.approx(64 * math.pi * R * R, rel=0.02)
    w2 = inputs.emulsion(n=2048, count=64, seed=5)
    assert np.array_equal(w["phi"], w2["phi"]) and np.array_equal(w["psi"], w2["psi"])


def test_emulsion3_workload():
    n, R = 64, 8.0
    w = inputs.emulsion3(n=n, count=8, R=R, seed=9)
    assert w["phi"].shape == (n, n, n) and len(w["droplets"]) == 8
    xi0 = inputs.interface_width(-0.001, 0.006, -0.05, 0.1)
    c = [(d["x"], d["y"], d["z"]) for d in w["droplets"]]
    dmin = min(min_image_dist(c[i], c[j], n) for i in range(8) for j in range(i))
    assert dmin >= 2 * R + 4 * xi0
    for centre, src in zip(c, w["sources"]):
        assert src[3] == R / 4
        assert min_image_dist(src[:3], centre, n) == pytest.approx(R - R / 4)
    assert np.abs(w["psi"] - 0.1).max() <= 0.005


def test_config_recipes():
    s = inputs.single_droplet()
    assert (s["nx"], s["ny"]) == (128, 128) and s["params"]["t_on"] == 1000
    assert s["params"]["M"] == 0.1 and s["params"]["tau"] == 1.0
    t = inputs.two_droplets(sep=80.0, offset=20.0)
    (a, b) = t["droplets"]
    assert (a["x"], a["y"], b["x"], b["y"]) == (216.0, 118.0, 296.0, 138.0)
    assert a["gx"] > 0 > b["gx"]  # each ramp points at the partner
    c = inputs.channel()
    assert c["params"]["flags"] == 16 and c["params"]["tau"] == 0.6
    assert (c["nx"], c["ny"]) == (512, 256)
