"""Hand-written adjoint of the coupled step (lbd_adjoint) against reverse-mode
autodiff of the independent torch FP64 restatement, against central finite
differences of the GPU forward, and for checkpoint-interval independence.

Loss: L = X_cm(T) - X_cm(0), the x displacement of the centre of mass of the
phi >= 0 region (Section 4); gradients with respect to psi(0) and B1.
Tolerances: FP64 adjoint vs torch autograd 1e-8 relative; vs central FD 1e-5;
FP32-forward adjoint vs FP64 FD 2e-2.  L is only piecewise smooth: the donor-cell
upwind choice switches where a face velocity changes sign, so central
differences carry an error from every switch that the +-h perturbation crosses
on top of an O(h^2) truncation error that is large here (at 64^2, 300 steps:
5e-4 relative at h = 1e-5, 1e-5 at h = 1e-6).  Below h ~ 3e-7 neither matters
and FP64 rounding of L (about 1e-14 absolute) is still far below the tolerance,
so the FD reference uses h = 2.5e-7.
"""
import numpy as np
import pytest
import torch

from oracle import torch_ref as T
from paper_1711_10984_gb300 import inputs, lbd
from paper_1711_10984_gb300.autograd import centroid_shift

pytestmark = pytest.mark.gpu

PAR = dict(a=-0.001, b=0.001, B0=0.006, B1=-0.05, M=0.5, D=0.1, tau=0.8, gamma=1.5e-3,
           c0=0.09, A0=2e-6, A_max=1e-4, t_on=20)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    lbd.load()


def case(n, seed=3):
    d = dict(x=n / 2 - 0.6, y=n / 2 + 0.3, R=n / 4, psi_mean=0.1, noise=0.01, gx=0.01)
    phi, psi = inputs.droplet_fields(n, n, [d], seed=seed)
    return d, phi, psi, [inputs.default_source(d, n, n)]


def gpu_grad(n, steps, K, prec=lbd.LBD_FP64, B1=PAR["B1"], psi=None):
    d, phi, psi0, src = case(n)
    psi = psi0 if psi is None else psi
    sim = lbd.Sim(n, n, precision=prec, sources=src, **dict(PAR, B1=B1))
    sim.set_fields(phi, psi)
    out = sim.adjoint(steps, K, n / 2)
    sim.close()
    return out


def gpu_loss(n, steps, psi, B1=PAR["B1"], prec=lbd.LBD_FP64):
    d, phi, _, src = case(n)
    sim = lbd.Sim(n, n, precision=prec, sources=src, **dict(PAR, B1=B1))
    sim.set_fields(phi, psi)
    x0 = sim.diagnostics(n / 2, n / 2)["cm_x"]
    sim.step(steps)
    x1 = sim.diagnostics(n / 2, n / 2)["cm_x"]
    sim.close()
    return x1 - x0


H = 2.5e-7


def central(f, h=H):
    return (f(h) - f(-h)) / (2 * h)


def test_adjoint_matches_torch_autograd():
    """32^2, 120 steps, source and sink switched on at step 20, checkpoints every
    7 steps (ragged last segment)."""
    n, steps = 32, 120
    d, phi, psi, src = case(n)
    L, dpsi, dB1 = gpu_grad(n, steps, 7)
    P = dict(PAR)
    psi_t = torch.tensor(psi, requires_grad=True)
    B1_t = torch.tensor(PAR["B1"], dtype=torch.float64, requires_grad=True)
    P["B1"] = B1_t
    phi_t = torch.tensor(phi)
    f, ph, c = T.run(P, phi_t, psi_t, steps, sources=src)
    Lt = T.centroid_x(ph, n / 2) - T.centroid_x(phi_t, n / 2)
    Lt.backward()
    assert L == pytest.approx(Lt.item(), rel=1e-10, abs=1e-12)
    g = psi_t.grad.numpy()
    assert np.abs(dpsi - g).max() <= 1e-8 * np.abs(g).max()
    assert dB1 == pytest.approx(B1_t.grad.item(), rel=1e-8)
    assert np.abs(g).max() > 0 and B1_t.grad.item() != 0


@pytest.mark.parametrize("nx,ny", [(40, 27), (20, 6)])
def test_adjoint_ragged_lattice(nx, ny):
    """Lattices that leave partial 32 x 8 blocks (and one smaller than a block)
    against torch autograd: the halo tiles of the fused reverse kernels wrap
    periodically through the partial blocks."""
    steps = 60
    d = dict(x=nx / 2 - 0.6, y=ny / 2 + 0.3, R=min(nx, ny) / 3, psi_mean=0.1, noise=0.01,
             gx=0.01)
    phi, psi = inputs.droplet_fields(nx, ny, [d], seed=5)
    src = [inputs.default_source(d, nx, ny)]
    sim = lbd.Sim(nx, ny, precision=lbd.LBD_FP64, sources=src, **PAR)
    sim.set_fields(phi, psi)
    L, dpsi, dB1 = sim.adjoint(steps, 9, nx / 2)
    sim.close()
    P = dict(PAR)
    psi_t = torch.tensor(psi, requires_grad=True)
    B1_t = torch.tensor(PAR["B1"], dtype=torch.float64, requires_grad=True)
    P["B1"] = B1_t
    phi_t = torch.tensor(phi)
    f, ph, c = T.run(P, phi_t, psi_t, steps, sources=src)
    Lt = T.centroid_x(ph, nx / 2) - T.centroid_x(phi_t, nx / 2)
    Lt.backward()
    assert L == pytest.approx(Lt.item(), rel=1e-10, abs=1e-12)
    g = psi_t.grad.numpy()
    assert np.abs(g).max() > 0
    assert np.abs(dpsi - g).max() <= 1e-8 * np.abs(g).max()
    assert dB1 == pytest.approx(B1_t.grad.item(), rel=1e-8, abs=1e-14)


def test_adjoint_matches_central_differences():
    """64^2, 300 steps: directional derivatives along seeded random directions
    in psi(0), single sites, and B1, against central differences of the FP64
    GPU forward."""
    n, steps = 64, 300
    d, phi, psi, src = case(n)
    L, dpsi, dB1 = gpu_grad(n, steps, 50)
    rng = np.random.default_rng(7)
    for k in range(3):
        v = rng.standard_normal((n, n))
        v /= np.abs(v).max()
        fd = central(lambda e: gpu_loss(n, steps, psi + e * v))
        ad = float((dpsi * v).sum())
        assert ad == pytest.approx(fd, rel=1e-5)
    # the largest-gradient sites
    for idx in np.argsort(np.abs(dpsi).ravel())[-2:]:
        e1 = np.zeros(n * n)
        e1[idx] = 1.0
        e1 = e1.reshape(n, n)
        fd = central(lambda e: gpu_loss(n, steps, psi + e * e1))
        assert dpsi.ravel()[idx] == pytest.approx(fd, rel=1e-5)
    fd = central(lambda e: gpu_loss(n, steps, psi, B1=PAR["B1"] + e))
    assert dB1 == pytest.approx(fd, rel=1e-5)


def test_checkpoint_interval_does_not_change_the_gradient():
    """Every checkpoint interval gives the same gradient bit for bit: one segment
    (90, 1000), even and odd intervals (2, 45, 13; the recompute of a segment runs
    on its own stream into one of two buffer sets, and the reverse sweeps of full
    segments replay graphs per set and adjoint-buffer parity), a partial last
    segment (13), one step per segment (1)."""
    n, steps = 48, 90
    outs = [gpu_grad(n, steps, K) for K in (1, 2, 13, 45, 90, 1000)]
    for L, dpsi, dB1 in outs[1:]:
        assert L == outs[0][0] and dB1 == outs[0][2]
        assert np.array_equal(dpsi, outs[0][1])


def test_adjoint_leaves_the_forward_state():
    n, steps = 40, 60
    d, phi, psi, src = case(n)
    a = lbd.Sim(n, n, sources=src, **PAR)
    a.set_fields(phi, psi)
    a.adjoint(steps, 16, n / 2, want_dpsi=False)
    b = lbd.Sim(n, n, sources=src, **PAR)
    b.set_fields(phi, psi)
    b.step(steps)
    assert a.t == b.t == steps
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)


def test_fp32_forward_adjoint_against_fp64_differences():
    """FP32 forward (shifted populations) with the FP32 reverse sweep: within 2e-2
    of FP64 central differences."""
    n, steps = 64, 300
    d, phi, psi, src = case(n)
    L, dpsi, dB1 = gpu_grad(n, steps, 50, prec=lbd.LBD_FP32)
    rng = np.random.default_rng(11)
    v = rng.standard_normal((n, n))
    v /= np.abs(v).max()
    fd = central(lambda e: gpu_loss(n, steps, psi + e * v))
    assert float((dpsi * v).sum()) == pytest.approx(fd, rel=2e-2)
    fdb = central(lambda e: gpu_loss(n, steps, psi, B1=PAR["B1"] + e))
    assert dB1 == pytest.approx(fdb, rel=2e-2)


def test_autograd_function():
    n, steps = 32, 80
    d, phi, psi, src = case(n)
    psi_t = torch.tensor(psi, requires_grad=True)
    B1_t = torch.tensor(PAR["B1"], dtype=torch.float64, requires_grad=True)
    P = {k: v for k, v in PAR.items() if k != "B1"}
    L = centroid_shift(psi_t, B1_t, phi0=phi, nsteps=steps, ckpt_every=10, refx=n / 2,
                       sources=src, params=P)
    (2.0 * L).backward()
    L2, dpsi, dB1 = gpu_grad(n, steps, 10)
    assert L.item() == pytest.approx(L2)
    assert np.allclose(psi_t.grad.numpy(), 2.0 * dpsi, rtol=0, atol=1e-12 * np.abs(dpsi).max())
    assert B1_t.grad.item() == pytest.approx(2.0 * dB1)


def test_config4_fp32_adjoint_against_fp64_differences():
    """The adjoint workload at its stated size: 256 x 256, one droplet R = 30 with
    a psi ramp, source and sink on from t = 0, FP32 forward (FP64 reductions),
    4000 steps, checkpoints every 100 steps (39 recomputed segments).  dL/dpsi0
    along three seeded directions and dL/dB1 within 2e-2 of central differences
    of the FP64 GPU forward (h = 2.5e-7, as above)."""
    n, steps, K = 256, 4000, 100
    d = dict(x=n / 2, y=n / 2, R=30.0, psi_mean=0.1, noise=0.01, gx=0.005)
    phi, psi = inputs.droplet_fields(n, n, [d], seed=4)
    par = dict(inputs.PAPER, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4, t_on=0)
    src = [inputs.default_source(d, n, n)]

    def loss(psi0, B1=par["B1"]):
        sim = lbd.Sim(n, n, precision=lbd.LBD_FP64, sources=src, **dict(par, B1=B1))
        sim.set_fields(phi, psi0)
        x0 = sim.diagnostics(n / 2, n / 2)["cm_x"]
        sim.step(steps)
        x1 = sim.diagnostics(n / 2, n / 2)["cm_x"]
        sim.close()
        return x1 - x0

    sim = lbd.Sim(n, n, precision=lbd.LBD_FP32, sources=src, **par)
    sim.set_fields(phi, psi)
    L, dpsi, dB1 = sim.adjoint(steps, K, n / 2)
    sim.close()
    assert np.isfinite(dpsi).all() and np.abs(dpsi).max() > 0
    rng = np.random.default_rng(41)
    for _ in range(3):
        v = rng.standard_normal((n, n))
        v /= np.abs(v).max()
        fd = central(lambda e: loss(psi + e * v))
        assert float((dpsi * v).sum()) == pytest.approx(fd, rel=2e-2)
    fdb = central(lambda e: loss(psi, B1=par["B1"] + e))
    assert dB1 == pytest.approx(fdb, rel=2e-2)
