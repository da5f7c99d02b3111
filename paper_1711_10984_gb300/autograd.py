"""torch.autograd binding of the hand-written adjoint (lbd_adjoint).

``centroid_shift(psi0, B1, phi0=..., nsteps=..., ...)`` returns the droplet
displacement L = X_cm(T) - X_cm(0) as a torch scalar whose backward gives
dL/dpsi0 and dL/dB1.  The forward run, the checkpoints and the reverse sweep
all happen inside the CUDA library in the forward call (the reverse sweep needs
only the forward's checkpoints, so both are done together); backward scales
the stored gradients by the incoming gradient.
"""
import numpy as np
import torch

from . import lbd


class CentroidShift(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0, B1, phi0, nsteps, ckpt_every, refx, precision, sources, params,
                stream):
        ny, nx = psi0.shape
        kw = dict(params)
        kw["B1"] = float(B1.detach().cpu())
        sim = lbd.Sim(nx, ny, precision=precision, sources=sources, stream=stream, **kw)
        try:
            sim.set_fields(np.asarray(phi0, dtype=np.float64),
                           psi0.detach().to("cpu", torch.float64).numpy())
            L, dpsi, dB1 = sim.adjoint(nsteps, ckpt_every, refx)
        finally:
            sim.close()
        ctx.save_for_backward(torch.from_numpy(dpsi).to(psi0.device, psi0.dtype),
                              torch.tensor(dB1, dtype=B1.dtype, device=B1.device))
        return torch.tensor(L, dtype=psi0.dtype, device=psi0.device)

    @staticmethod
    def backward(ctx, grad):
        dpsi, dB1 = ctx.saved_tensors
        return (grad * dpsi, grad * dB1) + (None,) * 8


def centroid_shift(psi0, B1, *, phi0, nsteps, ckpt_every=100, refx=None,
                   precision=lbd.LBD_FP64, sources=(), params=None, stream=None):
    """L = X_cm(nsteps) - X_cm(0) for a run started from (phi0, psi0) with the
    coupling B1; differentiable in psi0 (ny x nx tensor) and B1 (scalar tensor)."""
    ny, nx = psi0.shape
    refx = nx / 2.0 if refx is None else refx
    return CentroidShift.apply(psi0, B1, phi0, int(nsteps), int(ckpt_every), float(refx),
                               int(precision), list(sources), dict(params or {}), stream)
