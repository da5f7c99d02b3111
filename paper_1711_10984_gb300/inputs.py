"""Seeded synthetic initial fields for the droplet workloads.

This module builds the inputs both the CUDA path and the oracle start from:
phi (tanh droplets), psi (surfactant background plus per-droplet ramp and
noise) and the workload recipes with their seeds.  It holds none of the
method's arithmetic; it only lays out initial conditions.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014): draw k of the
stream with seed s is mix(s + (k+1) * 0x9E3779B97F4A7C15) where mix is the
published finaliser; a uniform in [0, 1) is (draw >> 11) * 2**-53.  Site k
(index y*nx + x) uses draw k.
"""
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, start=0):
    """Draws start .. start+count-1 of the SplitMix64 stream with this seed."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, count, start=0):
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def _min_image(d, L):
    return d - L * np.round(d / L)


def interface_width(a, B0, B1, psi_bg):
    """xi0 = sqrt(2 kappa / -a), kappa = B0 + B1 psi_bg: width of the tanh profile."""
    kappa = B0 + B1 * psi_bg
    return math.sqrt(2.0 * kappa / -a)


def droplet_fields(nx, ny, droplets, *, a=-0.001, b=0.001, B0=0.006, B1=-0.05,
                   psi_bg=0.1, xi=None, seed=0):
    """phi, psi of shape (ny, nx) for a set of droplets on a periodic lattice.

    droplets: iterable of dicts with keys x, y, R and optional psi_mean (default
    psi_bg), noise (half-width of the uniform noise inside the droplet, default 0),
    gx, gy (linear psi ramp: + gx*(x-xc)/R + gy*(y-yc)/R inside the droplet).
    phi = phi_eq tanh(max_k (R_k - r_k) / xi) with phi_eq = sqrt(-a/b), so phi > 0
    inside the droplets; r_k is the minimum-image distance to droplet k.
    """
    xi = interface_width(a, B0, B1, psi_bg) if xi is None else xi
    phieq = math.sqrt(-a / b)
    best = np.full((ny, nx), -np.inf)
    owner = np.full((ny, nx), -1)
    windows = []
    for k, d in enumerate(droplets):
        # tanh(-20) rounds to -1 in double: beyond R + 20 xi a droplet changes nothing
        half = d["R"] + 20.0 * xi
        xs = np.arange(math.floor(d["x"] - half), math.ceil(d["x"] + half) + 1)
        ys = np.arange(math.floor(d["y"] - half), math.ceil(d["y"] + half) + 1)
        if len(xs) >= nx:
            xs = np.arange(nx)
        if len(ys) >= ny:
            ys = np.arange(ny)
        xs, ys = xs % nx, ys % ny
        dx = _min_image(xs[None, :].astype(np.float64) - d["x"], nx)
        dy = _min_image(ys[:, None].astype(np.float64) - d["y"], ny)
        s = d["R"] - np.sqrt(dx * dx + dy * dy)
        sub = np.ix_(ys, xs)
        better = s > best[sub]
        best[sub] = np.where(better, s, best[sub])
        owner[sub] = np.where(better, k, owner[sub])
        windows.append((sub, dx, dy))
    phi = phieq * np.tanh(best / xi)
    psi = np.full((ny, nx), float(psi_bg))
    noise = 2.0 * uniform01(seed, nx * ny).reshape(ny, nx) - 1.0
    for k, d in enumerate(droplets):
        sub, dx, dy = windows[k]
        inside = (owner[sub] == k) & (best[sub] > 0)
        val = (d.get("psi_mean", psi_bg) + d.get("noise", 0.0) * noise[sub]
               + d.get("gx", 0.0) * dx / d["R"] + d.get("gy", 0.0) * dy / d["R"])
        psi[sub] = np.where(inside, val, psi[sub])
    return phi, psi


def default_source(d, nx=None, ny=None):
    """Source disk of radius R/4 internally tangent to droplet d on its +x side."""
    Rp = d["R"] / 4.0
    x = d["x"] + d["R"] - Rp
    if nx is not None:
        x = x % nx
    return (x, d["y"], Rp)


# ---------------------------------------------------------------- workloads
PAPER = dict(a=-0.001, b=0.001, B0=0.006, B1=-0.05, D=0.1, tau=1.0, M=0.1)


def single_droplet(n=128, R=20.0, seed=1):
    """One droplet, radius R, centred on an n x n lattice; psi = 0.1 with noise
    +-0.01 and a ramp 0.01 (x - xc)/R inside; passive for the first 1000 steps,
    then sink gamma = 1.5e-3 and the source schedule switch on."""
    d = dict(x=n / 2, y=n / 2, R=R, psi_mean=0.1, noise=0.01, gx=0.01)
    phi, psi = droplet_fields(n, n, [d], seed=seed)
    params = dict(PAPER, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4, t_on=1000)
    return dict(nx=n, ny=n, phi=phi, psi=psi, params=params,
                sources=[default_source(d, n, n)], droplets=[d])


def channel(nx=512, ny=256, R=32.0, B1=-0.05, seed=3):
    """Section 4's channel: one droplet of radius R at the centre of an nx x ny
    box between two plates (LBD_WALLS), psi = 0.1 with seeded noise, tau = 0.6,
    B0 = 0.006, B1 = +-0.05; sink gamma = 1.5e-3 and the source schedule on from
    the start, the source disk inside the droplet at its +x interface."""
    d = dict(x=nx / 2, y=ny / 2, R=R, psi_mean=0.1, noise=0.01, gx=0.0)
    phi, psi = droplet_fields(nx, ny, [d], seed=seed, B1=B1)
    params = dict(PAPER, B1=B1, tau=0.6, M=1.0, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4,
                  t_on=0, flags=16)
    return dict(nx=nx, ny=ny, phi=phi, psi=psi, params=params,
                sources=[default_source(d, nx, ny)], droplets=[d])


def ellipse_fields(n, R, eps, B1=0.0, a=-0.001, b=0.001, B0=0.006, psi_bg=0.1):
    """An area-preserving elliptical droplet (semi-axes R (1 + eps) along x and
    R / (1 + eps) along y) centred on an n x n lattice: phi = phi_eq
    tanh((1 - r_e) R / xi) with r_e the elliptical radius, psi = psi_bg."""
    xi = interface_width(a, B0, B1, psi_bg)
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    c = n / 2 - 0.5
    re = np.sqrt(((xx - c) / (R * (1 + eps))) ** 2 + ((yy - c) / (R / (1 + eps))) ** 2)
    phi = math.sqrt(-a / b) * np.tanh((1.0 - re) * R / xi)
    return phi, np.full((n, n), float(psi_bg))


def sphere_fields(nx, ny, nz, spheres, *, a=-0.001, b=0.001, B0=0.006, B1=-0.05, psi_bg=0.1,
                  noise=0.0, seed=0):
    """phi, psi of shape (nz, ny, nx) for droplets (x, y, z, R) on a periodic 3D
    lattice: phi = phi_eq tanh(max_k (R_k - r_k) / xi0), r_k the minimum-image
    distance; psi = psi_bg plus seeded uniform noise of half-width `noise`."""
    xi = interface_width(a, B0, B1, psi_bg)
    zz, yy, xx = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    best = np.full((nz, ny, nx), -np.inf)
    for (cx, cy, cz, R) in spheres:
        d = [_min_image(xx - cx, nx), _min_image(yy - cy, ny), _min_image(zz - cz, nz)]
        best = np.maximum(best, R - np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2))
    phi = math.sqrt(-a / b) * np.tanh(best / xi)
    u = 2.0 * uniform01(seed, nx * ny * nz).reshape(nz, ny, nx) - 1.0
    return phi, psi_bg + noise * u


def emulsion3(n=256, count=64, R=16.0, seed=9):
    """count spherical droplets of radius R at seeded non-overlapping positions
    (minimum centre distance 2R + 4 xi0, periodic) in an n^3 box; psi = 0.1
    with noise +-0.005; one source ball of radius R/4 inside each droplet,
    tangent to its +x surface."""
    xi0 = interface_width(PAPER["a"], PAPER["B0"], PAPER["B1"], 0.1)
    dmin = 2 * R + 4 * xi0
    centres = []
    k = 0
    while len(centres) < count and k < 100000:
        u = uniform01(seed + 7919 * k, 3) * n
        k += 1
        ok = True
        for c in centres:
            d = [_min_image(u[i] - c[i], n) for i in range(3)]
            if d[0] ** 2 + d[1] ** 2 + d[2] ** 2 < dmin ** 2:
                ok = False
                break
        if ok:
            centres.append((float(u[0]), float(u[1]), float(u[2])))
    spheres = [(x, y, z, R) for (x, y, z) in centres]
    phi, psi = sphere_fields(n, n, n, spheres, noise=0.005, seed=seed)
    srcs = [((x + R - R / 4) % n, y, z, R / 4) for (x, y, z) in centres]
    params = dict(PAPER, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4, t_on=0)
    return dict(nx=n, ny=n, nz=n, phi=phi, psi=psi, params=params, sources=srcs,
                droplets=[dict(x=x, y=y, z=z, R=R) for (x, y, z) in centres])


def two_droplets(nx=512, ny=256, R=25.0, sep=80.0, offset=0.0, seed=2):
    """Two droplets R on nx x ny, centres (nx/2 -+ sep/2, ny/2 -+ offset/2), each
    with a psi ramp pointing at its partner of seeded amplitude."""
    u = uniform01(seed ^ 0x5EED, 2)
    amp = 0.005 + 0.01 * u
    d1 = dict(x=nx / 2 - sep / 2, y=ny / 2 - offset / 2, R=R, psi_mean=0.1, noise=0.005,
              gx=float(amp[0]))
    d2 = dict(x=nx / 2 + sep / 2, y=ny / 2 + offset / 2, R=R, psi_mean=0.1, noise=0.005,
              gx=-float(amp[1]))
    phi, psi = droplet_fields(nx, ny, [d1, d2], seed=seed)
    s1 = default_source(d1, nx, ny)
    s2 = (d2["x"] - d2["R"] + d2["R"] / 4.0, d2["y"], d2["R"] / 4.0)
    params = dict(PAPER, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4, t_on=0)
    return dict(nx=nx, ny=ny, phi=phi, psi=psi, params=params, sources=[s1, s2],
                droplets=[d1, d2])


def emulsion(n=2048, count=64, R=25.0, seed=5):
    """count droplets of radius R at seeded non-overlapping positions on an
    n x n lattice (minimum centre distance 2R + 4 xi0, periodic), with seeded psi
    ramps of random direction."""
    xi0 = interface_width(PAPER["a"], PAPER["B0"], PAPER["B1"], 0.1)
    dmin = 2 * R + 4 * xi0
    centres = []
    k = 0
    while len(centres) < count:
        u = uniform01(seed, 2, start=2 * k)
        k += 1
        c = (float(u[0]) * n, float(u[1]) * n)
        ok = True
        for (x, y) in centres:
            dx = _min_image(c[0] - x, n)
            dy = _min_image(c[1] - y, n)
            if dx * dx + dy * dy < dmin * dmin:
                ok = False
                break
        if ok:
            centres.append(c)
        if k > 100000:
            raise RuntimeError("could not place droplets")
    ang = uniform01(seed ^ 0xA11CE, count) * 2 * math.pi
    drops, srcs = [], []
    for (x, y), th in zip(centres, ang):
        g = 0.01
        drops.append(dict(x=x, y=y, R=R, psi_mean=0.1, noise=0.005,
                          gx=g * math.cos(th), gy=g * math.sin(th)))
        Rp = R / 4
        srcs.append(((x + (R - Rp) * math.cos(th)) % n, (y + (R - Rp) * math.sin(th)) % n, Rp))
    phi, psi = droplet_fields(n, n, drops, seed=seed)
    params = dict(PAPER, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4, t_on=0)
    return dict(nx=n, ny=n, phi=phi, psi=psi, params=params, sources=srcs, droplets=drops)


def batch_sweep(count=256, seed=3, side_lo=128, side_hi=384):
    """Independent single-droplet instances: square lattices with sides uniform in
    [side_lo, side_hi], radii uniform in [15, 40] (at most a quarter of the side),
    |B1| log-uniform in [0.01, 0.05] (B1 < 0) and the psi asymmetry amplitude
    log-uniform in [1e-3, 2e-2]; source and sink on from step 0."""
    out = []
    for k in range(count):
        u = uniform01(seed * 1000003 + k, 6)
        n = int(side_lo + (side_hi - side_lo + 1) * u[0]) // 4 * 4
        n = max(side_lo, min(side_hi, n))
        R = min(15.0 + 25.0 * float(u[1]), n / 4.0)
        B1 = -math.exp(math.log(0.01) + (math.log(0.05) - math.log(0.01)) * float(u[2]))
        amp = math.exp(math.log(1e-3) + (math.log(2e-2) - math.log(1e-3)) * float(u[3]))
        d = dict(x=n / 2 + float(u[4]) - 0.5, y=n / 2 + float(u[5]) - 0.5, R=R, psi_mean=0.1,
                 noise=amp / 2, gx=amp)
        phi, psi = droplet_fields(n, n, [d], B1=B1, seed=seed * 7919 + k)
        params = dict(PAPER, B1=B1, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4, t_on=0)
        out.append(dict(nx=n, ny=n, phi=phi, psi=psi, params=params,
                        sources=[default_source(d, n, n)], droplets=[d]))
    return out