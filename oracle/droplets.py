"""Per-droplet tracking and the squirmer fit of Section 4 (Eq. 21), plain numpy.

TEST INFRASTRUCTURE ONLY (imported by tests/ and the bench's CPU leg, never by
the product package).  Readings (the paper gives the formulas, not the
discretisation):

* Centre of mass, Section 4: r_CM = sum phi r / sum phi over the sites with
  phi >= 0.  With several droplets every such site belongs to the nearest
  reference point (minimum image in x, and in y unless plates bound the
  lattice; ties to the lower index); its displacement from that reference is
  taken as the minimum image, and the centre is reference + mean displacement,
  wrapped into the lattice.  The droplet velocity U is the phi-weighted mean
  fluid velocity over the same sites.
* Polar velocity on the interface, Eq. (21): the phi = 0 contour is sampled
  where phi changes sign along a lattice link (x to x+1, y to y+1; no link
  through a plate), the point and its velocity interpolated linearly along the
  link.  Each point belongs to the nearest droplet centre.  In the droplet
  frame (velocity minus U), with theta measured from the swimming direction
  e = U / |U| (e = x when U = 0) and counted towards e_perp = z x e, the polar
  component is u_theta = (u - U) . (-sin(theta) e + cos(theta) e_perp).
* Fit: least squares of u_theta(theta_p) = b1 sin(theta_p) + (1/2) b2 sin(2 theta_p)
  over the points of the droplet, all points weighted equally; beta = b2 / b1.
"""
import numpy as np


def _min_image(d, n):
    return d - n * np.round(d / n)


def _nearest(px, py, refs, nx, ny, wrap_y):
    best = np.full(px.shape, -1, dtype=np.int64)
    bestd = np.full(px.shape, np.inf)
    for k, (rx, ry) in enumerate(refs):
        dx = _min_image(px - rx, nx)
        dy = _min_image(py - ry, ny) if wrap_y else py - ry
        d2 = dx * dx + dy * dy
        take = d2 < bestd
        best[take] = k
        bestd[take] = d2[take]
    return best


def droplets(phi, ux, uy, refs, walls=False):
    """Per droplet: dict(x, y, mass, ux, uy, sites)."""
    ny, nx = phi.shape
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    mask = phi >= 0.0
    px, py, w = xx[mask], yy[mask], phi[mask]
    vx, vy = ux[mask], uy[mask]
    lab = _nearest(px, py, refs, nx, ny, not walls)
    out = []
    for k, (rx, ry) in enumerate(refs):
        sel = lab == k
        m = float(np.sum(w[sel]))
        dx = _min_image(px[sel] - rx, nx)
        dy = _min_image(py[sel] - ry, ny) if not walls else py[sel] - ry
        if m > 0:
            cx = (rx + np.sum(w[sel] * dx) / m) % nx
            cy = ry + np.sum(w[sel] * dy) / m
            cy = cy % ny if not walls else cy
            u = (float(np.sum(w[sel] * vx[sel]) / m), float(np.sum(w[sel] * vy[sel]) / m))
        else:
            cx, cy, u = np.nan, np.nan, (np.nan, np.nan)
        out.append(dict(x=float(cx), y=float(cy), mass=m, ux=u[0], uy=u[1], sites=int(sel.sum())))
    return out


def interface_points(phi, ux, uy, walls=False):
    """phi = 0 crossings on the links: arrays x, y, u_x, u_y."""
    ny, nx = phi.shape
    xs, ys, us, vs = [], [], [], []
    for (ax, ay) in ((1, 0), (0, 1)):
        for y in range(ny):
            y2 = y + ay
            if y2 >= ny:
                if walls:
                    continue
                y2 -= ny
            for x in range(nx):
                x2 = (x + ax) % nx
                a, b = phi[y, x], phi[y2, x2]
                if (a >= 0.0) == (b >= 0.0):
                    continue
                t = a / (a - b)
                xs.append(x + t * ax)
                ys.append(y + t * ay)
                us.append((1 - t) * ux[y, x] + t * ux[y2, x2])
                vs.append((1 - t) * uy[y, x] + t * uy[y2, x2])
    return np.array(xs), np.array(ys), np.array(us), np.array(vs)


def squirmer(phi, ux, uy, drops, walls=False):
    """Per droplet: dict(b1, b2, points) from the least-squares fit of Eq. (21)."""
    ny, nx = phi.shape
    px, py, pu, pv = interface_points(phi, ux, uy, walls)
    centres = [(d["x"], d["y"]) for d in drops]
    lab = _nearest(px, py, centres, nx, ny, not walls)
    out = []
    for k, d in enumerate(drops):
        sel = lab == k
        U = np.array([d["ux"], d["uy"]])
        sp = np.hypot(U[0], U[1])
        e = U / sp if sp > 0 else np.array([1.0, 0.0])
        ep = np.array([-e[1], e[0]])
        dx = _min_image(px[sel] - d["x"], nx)
        dy = _min_image(py[sel] - d["y"], ny) if not walls else py[sel] - d["y"]
        r = np.hypot(dx, dy)
        c = (dx * e[0] + dy * e[1]) / r          # cos theta
        s = (dx * ep[0] + dy * ep[1]) / r        # sin theta
        wx, wy = pu[sel] - U[0], pv[sel] - U[1]
        ut = wx * (-s * e[0] + c * ep[0]) + wy * (-s * e[1] + c * ep[1])
        # design matrix columns sin(theta) and sin(2 theta) / 2
        A = np.stack([s, s * c], axis=1)
        if len(ut) >= 2:
            coef = np.linalg.lstsq(A, ut, rcond=None)[0]
            out.append(dict(b1=float(coef[0]), b2=float(coef[1]), points=int(sel.sum())))
        else:
            out.append(dict(b1=np.nan, b2=np.nan, points=int(sel.sum())))
    return out
