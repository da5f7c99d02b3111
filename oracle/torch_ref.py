"""Second, independent FP64 restatement of the coupled step, in vectorised torch.

TEST INFRASTRUCTURE ONLY.  Written separately from ``lbd_oracle.c`` (whole-field
``torch.roll`` shifts instead of per-site loops, stencils written with their
explicit coefficients, fluxes shared between neighbouring faces by a roll) so
that a transcription slip in either one shows up as a disagreement.  Because
every operation is a differentiable torch op on CPU float64 tensors, it is
also the reverse-mode (autograd) reference for the hand-written adjoint.

Follows arXiv 1711.10984, Section 2 with the readings stated in the C oracle's
header (factor 1/2 in Eq. (12); mobility M in Eq. (18); conservative donor-cell
advection for Eqs. (16)-(17); log-free form of c grad mu_c; isotropic D2Q9
stencils; force -> LB -> advection -> diffusion order).
"""
import math

import torch

# D2Q9 velocities and weights (Section 2.2), listed independently of the C file.
E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
WGT = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


def sh(g, dx, dy):
    """Field whose value at (x, y) is g at (x+dx, y+dy), periodic; g is [..., ny, nx]."""
    return torch.roll(g, shifts=(-dy, -dx), dims=(-2, -1))


def ddx(g):
    axis = sh(g, 1, 0) - sh(g, -1, 0)
    diag = (sh(g, 1, 1) - sh(g, -1, 1)) + (sh(g, 1, -1) - sh(g, -1, -1))
    return axis / 3.0 + diag / 12.0


def ddy(g):
    axis = sh(g, 0, 1) - sh(g, 0, -1)
    diag = (sh(g, 1, 1) - sh(g, 1, -1)) + (sh(g, -1, 1) - sh(g, -1, -1))
    return axis / 3.0 + diag / 12.0


def lap9(g):
    axis = sh(g, 1, 0) + sh(g, -1, 0) + sh(g, 0, 1) + sh(g, 0, -1) - 4.0 * g
    diag = sh(g, 1, 1) + sh(g, -1, 1) + sh(g, -1, -1) + sh(g, 1, -1) - 4.0 * g
    return (2.0 / 3.0) * axis + (1.0 / 6.0) * diag


def div_k_grad(k, g):
    """div(k grad g) as a sum over the 8 links with the link-mean coefficient."""
    out = torch.zeros_like(g)
    for (ex, ey), w in zip(E[1:], WGT[1:]):
        out = out + 6.0 * w * 0.5 * (k + sh(k, ex, ey)) * (sh(g, ex, ey) - g)
    return out


def mu_phi(P, phi, cube, c):
    """Eq. (3): a phi + b cube - B(c) lap phi - B1 grad phi . grad c."""
    return (P["a"] * phi + P["b"] * cube - (P["B0"] + P["B1"] * c) * lap9(phi)
            - P["B1"] * (ddx(phi) * ddx(c) + ddy(phi) * ddy(c)))


def m_part(P, phi):
    """(B1/2)|grad phi|^2, the gradient part of mu_c in Eq. (5)."""
    return 0.5 * P["B1"] * (ddx(phi) ** 2 + ddy(phi) ** 2)


def force(P, phi, c):
    """Eq. (14) with c grad mu_c = grad c + c grad m."""
    mu = mu_phi(P, phi, phi ** 3, c)
    m = m_part(P, phi)
    Fx = -phi * ddx(mu) - (ddx(c) + c * ddx(m))
    Fy = -phi * ddy(mu) - (ddy(c) + c * ddy(m))
    if "fx" in P:
        Fx = Fx + P["fx"]
        Fy = Fy + P["fy"]
    return Fx, Fy


def moments(f, Fx, Fy):
    n = f.sum(0)
    jx = sum(ex * f[i] for i, (ex, ey) in enumerate(E) if ex)
    jy = sum(ey * f[i] for i, (ex, ey) in enumerate(E) if ey)
    return n, (jx + 0.5 * Fx) / n, (jy + 0.5 * Fy) / n


def lb(P, f, Fx, Fy):
    """Eqs. (10)-(13): returns streamed populations and the velocity u^n."""
    n, ux, uy = moments(f, Fx, Fy)
    usq = ux * ux + uy * uy
    pref = 1.0 - 0.5 / P["tau"]
    out = []
    for i, ((ex, ey), w) in enumerate(zip(E, WGT)):
        eu = ex * ux + ey * uy
        feq = w * n * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq)
        eF = ex * Fx + ey * Fy
        uF = ux * Fx + uy * Fy
        Fi = pref * w * (3.0 * (eF - uF) + 9.0 * eu * eF)
        post = f[i] - (f[i] - feq) / P["tau"] + Fi
        out.append(sh(post, -ex, -ey))   # value at x comes from x - e_i
    return torch.stack(out), ux, uy


def advect(g, ux, uy):
    """Donor-cell flux form: face (x, x+1) flux = u_f * upwind g."""
    ufx = 0.5 * (ux + sh(ux, 1, 0))
    fe = torch.where(ufx > 0, ufx * g, ufx * sh(g, 1, 0))
    ufy = 0.5 * (uy + sh(uy, 0, 1))
    fn = torch.where(ufy > 0, ufy * g, ufy * sh(g, 0, 1))
    return g - ((fe - sh(fe, -1, 0)) + (fn - sh(fn, 0, -1)))


def source_mask(nx, ny, sources, dtype=torch.float64):
    X = torch.arange(nx, dtype=dtype).view(1, nx).expand(ny, nx)
    Y = torch.arange(ny, dtype=dtype).view(ny, 1).expand(ny, nx)
    mask = torch.zeros(ny, nx, dtype=torch.bool)
    for (sx, sy, R) in sources:
        dx = X - sx
        dy = Y - sy
        dx = dx - nx * torch.round(dx / nx)
        dy = dy - ny * torch.round(dy / ny)
        mask |= dx * dx + dy * dy <= R * R
    return mask.to(dtype)


def activity(P, t):
    if t < P["t_on"]:
        return 0.0, 0.0
    return min(P["A0"] * (t - P["t_on"]), P["A_max"]), P["gamma"]


def step(P, f, phi, c, t, theta):
    """One coupled step n -> n+1 (force, LB, advection, diffusion)."""
    A, gamma = activity(P, t)
    Fx, Fy = force(P, phi, c)
    f2, ux, uy = lb(P, f, Fx, Fy)
    if "ux0" in P:
        ux = torch.full_like(ux, P["ux0"])
        uy = torch.full_like(uy, P["uy0"])
    phs = advect(phi, ux, uy)
    cs = advect(c, ux, uy)
    mus = mu_phi(P, phs, phi ** 3, cs)
    phi2 = phs + P["M"] * lap9(mus)
    ms = m_part(P, phs)
    c2 = cs + (P["D"] * (lap9(cs) + div_k_grad(cs, ms)) - gamma * (cs - P["c0"]) + A * theta)
    return f2, phi2, c2


def equilibrium(n, ux, uy):
    usq = ux * ux + uy * uy
    return torch.stack([w * n * (1.0 + 3.0 * (ex * ux + ey * uy) + 4.5 * (ex * ux + ey * uy) ** 2
                                 - 1.5 * usq) for (ex, ey), w in zip(E, WGT)])


def run(P, phi, c, nsteps, sources=(), rho=None, ux=None, uy=None, t0=0):
    ny, nx = phi.shape
    rho = torch.ones_like(phi) if rho is None else rho
    ux = torch.zeros_like(phi) if ux is None else ux
    uy = torch.zeros_like(phi) if uy is None else uy
    f = equilibrium(rho, ux, uy)
    theta = source_mask(nx, ny, sources)
    for k in range(nsteps):
        f, phi, c = step(P, f, phi, c, t0 + k, theta)
    return f, phi, c


def fields(P, f, phi, c):
    Fx, Fy = force(P, phi, c)
    n, ux, uy = moments(f, Fx, Fy)
    return n, ux, uy


def centroid_x(phi, refx):
    """x centre of mass over phi >= 0 (Section 4), minimum image about refx."""
    ny, nx = phi.shape
    X = torch.arange(nx, dtype=phi.dtype).view(1, nx).expand(ny, nx)
    dx = X - refx
    dx = dx - nx * torch.floor(dx / nx + 0.5)
    w = torch.where(phi >= 0, phi, torch.zeros_like(phi))
    return refx + (w * dx).sum() / w.sum()


def sigma_flat_closed_form(a, b, kappa):
    """Interface tension of a flat phi^4 interface with constant stiffness kappa:
    sigma = sqrt(-8 kappa a^3 / (9 b^2))."""
    return math.sqrt(-8.0 * kappa * a ** 3 / (9.0 * b * b))
