"""Batched instances (one persistent launch per step, CUDA-graph replay): every
instance matches the same instance run on its own, bit for bit, and the
batched FP64 path matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    lbd.load()


SIZES = [(64, 64), (100, 80), (130, 130), (37, 50), (200, 120)]


def instances():
    out = []
    for k, (nx, ny) in enumerate(SIZES):
        d = dict(x=nx / 2 + 0.3 * k, y=ny / 2 - 0.2, R=min(nx, ny) / 4, psi_mean=0.1,
                 noise=0.01, gx=0.002 * (k + 1))
        phi, psi = inputs.droplet_fields(nx, ny, [d], seed=100 + k)
        kw = dict(a=-0.001, b=0.001, B0=0.006, B1=-0.008 * (k + 1), M=0.3 + 0.1 * k, D=0.1,
                  tau=0.7 + 0.1 * k, gamma=1.5e-3, c0=0.09, A0=1e-6 * (k + 1), A_max=1e-4,
                  t_on=30 * k)
        out.append((nx, ny, phi, psi, [inputs.default_source(d, nx, ny)], kw))
    return out


def make_batch(prec, tile=(118, 64)):
    inst = instances()
    params = [lbd.make_params(prec, src, **kw) for (_, _, _, _, src, kw) in inst]
    b = lbd.Batch([(nx, ny) for (nx, ny, *_r) in inst], params)
    b.set_tile(*tile)
    for k, (nx, ny, phi, psi, src, kw) in enumerate(inst):
        b.set_fields(k, phi, psi)
    return b, inst


def alone(prec, inst, steps, tile=(118, 64)):
    outs = []
    for (nx, ny, phi, psi, src, kw) in inst:
        s = lbd.Sim(nx, ny, precision=prec, sources=src, **kw)
        s.set_tile(*tile)
        s.set_fields(phi, psi)
        s.step(steps)
        outs.append(s.fields())
        s.close()
    return outs


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
@pytest.mark.parametrize("tile", [(118, 64), (246, 32)])
def test_batch_equals_instances_alone(prec, tile):
    b, inst = make_batch(prec, tile)
    b.step(101)   # one graph replay of 100 steps + 1 direct step (odd parity)
    b.step(149)   # graph replays from the other parity + remainder
    ref = alone(prec, inst, 250, tile)
    for k in range(len(inst)):
        for a, r in zip(b.fields(k), ref[k]):
            assert np.array_equal(a, r), k
    assert b.t == 250
    b.close()


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
def test_batch_with_plates_equals_instances_alone(prec):
    """A batch mixing periodic instances and instances between plates
    (LBD_WALLS): each one still equals the same instance run on its own."""
    inst = instances()
    walls = [k % 2 == 1 for k in range(len(inst))]
    params = [lbd.make_params(prec, src, flags=lbd.LBD_WALLS if wl else 0, **kw)
              for wl, (_, _, _, _, src, kw) in zip(walls, inst)]
    b = lbd.Batch([(nx, ny) for (nx, ny, *_r) in inst], params)
    b.set_tile(118, 32)
    for k, (nx, ny, phi, psi, src, kw) in enumerate(inst):
        b.set_fields(k, phi, psi)
    b.step(130)
    for k, (nx, ny, phi, psi, src, kw) in enumerate(inst):
        s = lbd.Sim(nx, ny, precision=prec, sources=src,
                    flags=lbd.LBD_WALLS if walls[k] else 0, **kw)
        s.set_tile(118, 32)
        s.set_fields(phi, psi)
        s.step(130)
        for a, r in zip(b.fields(k), s.fields()):
            assert np.array_equal(a, r), k
        s.close()
    b.close()


def test_graph_and_direct_launches_agree():
    b1, _ = make_batch(lbd.LBD_FP32)
    b2, _ = make_batch(lbd.LBD_FP32)
    b1.step(200)
    for _ in range(200):
        b2.step(1)
    for k in range(len(SIZES)):
        for a, r in zip(b1.fields(k), b2.fields(k)):
            assert np.array_equal(a, r)


def test_batch_fp64_matches_oracle():
    b, inst = make_batch(lbd.LBD_FP64)
    b.step(120)
    for k, (nx, ny, phi, psi, src, kw) in enumerate(inst):
        ref = oracle.State(oracle.Params(nx, ny, sources=src, **kw), phi, psi).step(120).fields()
        for a, r in zip(b.fields(k), ref):
            assert np.abs(a - r).max() <= 1e-10 * max(np.abs(r).max(), 1e-300)


def test_batch_autotune_keeps_state():
    b1, _ = make_batch(lbd.LBD_FP32)
    b2, _ = make_batch(lbd.LBD_FP32)
    b1.step(10)
    tile = b1.autotune(2)
    assert tile[0] in (118, 246)
    b1.set_tile(118, 64)
    b1.step(40)
    b2.step(50)
    for k in range(len(SIZES)):
        for a, r in zip(b1.fields(k), b2.fields(k)):
            assert np.array_equal(a, r)


def test_sweep_recipe():
    w = inputs.batch_sweep(count=8)
    for x in w:
        assert 128 <= x["nx"] <= 384 and x["nx"] % 4 == 0
        assert -0.05 <= x["params"]["B1"] <= -0.01
        assert 15 <= x["droplets"][0]["R"] <= 40


SIZES4 = [(64, 64), (100, 80), (132, 132), (36, 52), (200, 120)]  # all 4k wide


def instances4():
    out = []
    for k, (nx, ny) in enumerate(SIZES4):
        d = dict(x=nx / 2 + 0.3 * k, y=ny / 2 - 0.2, R=min(nx, ny) / 4, psi_mean=0.1,
                 noise=0.01, gx=0.002 * (k + 1))
        phi, psi = inputs.droplet_fields(nx, ny, [d], seed=200 + k)
        kw = dict(a=-0.001, b=0.001, B0=0.006, B1=-0.008 * (k + 1), M=0.3 + 0.1 * k, D=0.1,
                  tau=0.7 + 0.1 * k, gamma=1.5e-3, c0=0.09, A0=1e-6 * (k + 1), A_max=1e-4,
                  t_on=30 * k)
        out.append((nx, ny, phi, psi, [inputs.default_source(d, nx, ny)], kw))
    return out


@pytest.mark.parametrize("tile", [(116, 64), (116, 32)])
def test_staged_kernel_batch_equals_instances_alone(tile):
    """FP32 batch on the 16-byte staged stripe kernel (4k-wide instances), graph
    replays of both parities: each instance equals itself run alone in the same
    launch shape, and a batch of such instances starts on this kernel."""
    inst = instances4()
    params = [lbd.make_params(lbd.LBD_FP32, src, **kw) for (_, _, _, _, src, kw) in inst]
    b = lbd.Batch([(nx, ny) for (nx, ny, *_r) in inst], params)
    assert b.tile == (116, 64)
    b.set_tile(*tile)
    for k, (nx, ny, phi, psi, src, kw) in enumerate(inst):
        b.set_fields(k, phi, psi)
    b.step(101)
    b.step(149)
    ref = alone(lbd.LBD_FP32, inst, 250, tile)
    for k in range(len(inst)):
        for a, r in zip(b.fields(k), ref[k]):
            assert np.array_equal(a, r), k
    b.close()


def test_staged_kernel_batch_with_plates():
    """Under bx 116 the periodic instances run the staged kernel and those
    between plates the 118-column stripe kernel; each equals its own run."""
    inst = instances4()
    walls = [k % 2 == 1 for k in range(len(inst))]
    params = [lbd.make_params(lbd.LBD_FP32, src, flags=lbd.LBD_WALLS if wl else 0, **kw)
              for wl, (_, _, _, _, src, kw) in zip(walls, inst)]
    b = lbd.Batch([(nx, ny) for (nx, ny, *_r) in inst], params)
    b.set_tile(116, 32)
    for k, (nx, ny, phi, psi, src, kw) in enumerate(inst):
        b.set_fields(k, phi, psi)
    b.step(130)
    for k, (nx, ny, phi, psi, src, kw) in enumerate(inst):
        s = lbd.Sim(nx, ny, precision=lbd.LBD_FP32, sources=src,
                    flags=lbd.LBD_WALLS if walls[k] else 0, **kw)
        s.set_tile(118 if walls[k] else 116, 32)
        s.set_fields(phi, psi)
        s.step(130)
        for a, r in zip(b.fields(k), s.fields()):
            assert np.array_equal(a, r), k
        s.close()
    b.close()


def test_staged_kernel_rejected_for_unsupported_batches():
    """bx 116 needs FP32 and 4k-wide periodic instances."""
    b, _ = make_batch(lbd.LBD_FP32)           # holds a 37-wide instance
    with pytest.raises(lbd.LbdError):
        b.set_tile(116, 64)
    assert b.tile == (118, 64)
    b.close()
    inst = instances4()
    params = [lbd.make_params(lbd.LBD_FP64, src, **kw) for (_, _, _, _, src, kw) in inst]
    b = lbd.Batch([(nx, ny) for (nx, ny, *_r) in inst], params)
    with pytest.raises(lbd.LbdError):
        b.set_tile(116, 64)
    b.close()
