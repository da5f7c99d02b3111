"""Parity at the bench's full size: the 2048 x 2048 emulsion (64 droplets R = 25
with seeded psi ramps, 64 sources, sink on), in the launch shape the bench
times (the autotuner's choice for this lattice) and in every stripe shape it
chooses from; and the bench's walls leg, the same emulsion between bounce-back
plates at y = -1/2 and 2047.5.

The GPU runs from the seeded initial state into developed flow; its state then
(pre-collision populations, phi, psi, t) is handed to the FP64 oracle, and both
advance a few more steps.  The whole lattice is compared, not samples: the C
oracle takes a 2048^2 step in well under a second on the host's cores.
Tolerances: FP64 max relative error 1e-10 per field and for the populations;
FP32 (shifted populations) phi, psi and u within 1e-4 absolute.
"""
import numpy as np
import pytest

import oracle
from paper_1711_10984_gb300 import autotune, inputs, lbd

pytestmark = pytest.mark.gpu

N = 2048
LEAD, STEPS = 300, 3


@pytest.fixture(scope="module")
def work():
    from paper_1711_10984_gb300 import build
    build.build()
    import oracle.build
    oracle.build.build()
    lbd.load()
    return inputs.emulsion(n=N, count=64, seed=5)


def advance_both(w, prec, tile, walls=False):
    sim = lbd.Sim(N, N, precision=prec, sources=w["sources"],
                  flags=lbd.LBD_WALLS if walls else 0, **w["params"])
    if tile == "bench":
        import torch
        tile = autotune.tune(sim, torch.cuda.get_device_name())
    else:
        sim.set_tile(*tile)
    sim.set_fields(w["phi"], w["psi"])
    sim.step(LEAD)
    _, _, _, phi, psi = sim.fields()
    ref = oracle.State(oracle.Params(N, N, sources=w["sources"], flags=oracle.WALLS if walls else 0,
                                     **w["params"]), phi, psi, t=sim.t)
    ref.f[...] = sim.populations()
    sim.step(STEPS)
    ref.step(STEPS)
    out = (sim.fields(), sim.populations(), ref.fields(), ref.f.copy(), tuple(tile))
    sim.close()
    return out


@pytest.mark.parametrize("tile", ["bench", (118, 128), (246, 64)], ids=str)
def test_fp64_full_size(work, tile):
    g, gf, r, rf, used = advance_both(work, lbd.LBD_FP64, tile)
    for a, b, name in zip(g, r, ["rho", "ux", "uy", "phi", "psi"]):
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err <= 1e-10, (name, used, err)
    assert np.abs(gf - rf).max() / np.abs(rf).max() <= 1e-10
    assert np.abs(g[1]).max() > 1e-8  # the flow has developed: every term is exercised


@pytest.mark.parametrize("tile", ["bench", (118, 64), (246, 64), (116, 64), (116, 32)], ids=str)
def test_fp32_full_size(work, tile):
    g, _, r, _, used = advance_both(work, lbd.LBD_FP32, tile)
    for k in (1, 2, 3, 4):  # ux, uy, phi, psi
        assert np.abs(g[k] - r[k]).max() <= 1e-4, (k, used)
    assert np.abs(g[0] - r[0]).max() <= 1e-5


@pytest.mark.parametrize("prec,tile", [(lbd.LBD_FP32, "bench"), (lbd.LBD_FP64, (118, 64))],
                         ids=["fp32-bench", "fp64-118x64"])
def test_walls_full_size(work, prec, tile):
    g, gf, r, rf, used = advance_both(work, prec, tile, walls=True)
    if prec == lbd.LBD_FP64:
        for a, b in zip(g, r):
            assert np.abs(a - b).max() / np.abs(b).max() <= 1e-10, used
        assert np.abs(gf - rf).max() / np.abs(rf).max() <= 1e-10
    else:
        for k in (1, 2, 3, 4):
            assert np.abs(g[k] - r[k]).max() <= 1e-4, (k, used)
