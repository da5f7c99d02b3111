"""Run-time failure detection, tested without faulting the GPU.

* A state driven past the stability limit of Section 4 (B(psi) <= 0 somewhere:
  the droplet breaks up) through the parameters: the run-time checks of
  lbd_set_check report LBD_EUNSTABLE, steps are refused until the state is
  replaced, and lbd_diagnostics returns the same verdict with its values.
* A state driven to Inf/NaN by an absurd body force (IEEE arithmetic, no
  fault): the checks report LBD_ENONFINITE.
* Device-allocation failures made on the host by the lbd_debug_fail_alloc
  hook: every allocation of lbd_create, and the on-demand allocations of the
  other entry points, return LBD_ENOMEM and leave the context usable (or, for
  lbd_create, no context at all).
"""
import ctypes

import numpy as np
import pytest

from paper_1711_10984_gb300 import inputs, lbd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1711_10984_gb300 import build
    build.build()
    lbd.load()
    yield
    lbd.load().lbd_debug_fail_alloc(0)


def droplet_state(n=64, seed=3):
    d = dict(x=n / 2, y=n / 2, R=n / 5, psi_mean=0.1, noise=0.01, gx=0.005)
    return inputs.droplet_fields(n, n, [d], seed=seed)


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
def test_checks_report_instability(prec):
    n = 64
    phi, psi = droplet_state(n)
    sim = lbd.Sim(n, n, precision=prec, tau=0.8, M=0.5)
    sim.set_fields(phi, psi)
    sim.set_check(10)
    sim.step(30)
    sim.synchronize()                      # stable: every check passes
    # B1 = -0.07 makes B = B0 + B1 psi = 0.006 - 0.007 < 0 at psi = 0.1
    sim.set_params(precision=prec, tau=0.8, M=0.5, B1=-0.07)
    try:
        sim.step(20)                       # the checks are queued; verdicts follow
    except lbd.LbdError as e:
        assert e.code == lbd.LBD_EUNSTABLE
    with pytest.raises(lbd.LbdError) as e:
        sim.synchronize()
    assert e.value.code == lbd.LBD_EUNSTABLE and "min B" in str(e.value)
    with pytest.raises(lbd.LbdError) as e:
        sim.step(1)                        # refused until the state is replaced
    assert e.value.code == lbd.LBD_EUNSTABLE
    d = sim.diagnostics(n / 2, n / 2)
    assert d["status"] == lbd.LBD_EUNSTABLE and d["min_B"] <= 0
    with pytest.raises(lbd.LbdError):
        sim.diagnostics(n / 2, n / 2, check=True)
    sim.set_params(precision=prec, tau=0.8, M=0.5)
    sim.set_fields(phi, psi)               # a new state clears the verdict
    sim.step(20)
    sim.synchronize()
    assert sim.diagnostics(n / 2, n / 2)["status"] == lbd.LBD_OK
    sim.close()


@pytest.mark.parametrize("prec", [lbd.LBD_FP64, lbd.LBD_FP32])
def test_checks_report_nonfinite(prec):
    n = 32
    phi, psi = droplet_state(n)
    sim = lbd.Sim(n, n, precision=prec, flags=lbd.LBD_BODY_FORCE, fx=1e300 if prec == 0 else 1e30)
    sim.set_fields(phi, psi)
    sim.set_check(1)
    try:
        sim.step(6)
    except lbd.LbdError as e:
        assert e.code == lbd.LBD_ENONFINITE
    with pytest.raises(lbd.LbdError) as e:
        sim.synchronize()
    assert e.value.code == lbd.LBD_ENONFINITE and "non-finite" in str(e.value)
    d = sim.diagnostics(1.0, 1.0)
    assert d["status"] == lbd.LBD_ENONFINITE and d["nonfinite"] > 0
    sim.close()


def test_checks_off_by_default_and_cheap_state_unchanged():
    """Checks only read the state: a run with checks every step ends in the
    same state as one without."""
    n = 48
    phi, psi = droplet_state(n)
    outs = []
    for every in (0, 1):
        sim = lbd.Sim(n, n, precision=lbd.LBD_FP32, tau=0.8, M=0.5)
        sim.set_fields(phi, psi)
        sim.set_check(every)
        sim.step(40)
        sim.synchronize()
        outs.append(sim.fields())
        sim.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def _create(n=32, prec=lbd.LBD_FP32):
    p = lbd.make_params(prec)
    g = lbd.lbd_grid(n, n)
    h = ctypes.c_void_p()
    return lbd.load().lbd_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h)), h


def test_create_allocation_failures():
    L = lbd.load()
    created = 0
    for nth in range(1, 16):
        L.lbd_debug_fail_alloc(nth)
        rc, h = _create()
        if rc == lbd.LBD_OK:               # nth is past the allocations of lbd_create
            L.lbd_destroy(h)
            created += 1
            continue
        assert rc == lbd.LBD_ENOMEM, nth
        assert not h.value, nth             # no context on failure
    L.lbd_debug_fail_alloc(0)
    assert created >= 1
    rc, h = _create()
    assert rc == lbd.LBD_OK
    L.lbd_destroy(h)


def test_on_demand_allocation_failures_leave_context_usable():
    L = lbd.load()
    n = 32
    phi, psi = droplet_state(n)
    sim = lbd.Sim(n, n, precision=lbd.LBD_FP32, tau=0.8, M=0.5)
    calls = [
        ("set_fields", lambda: sim.set_fields(phi, psi)),
        ("populations", lambda: sim.populations()),
        ("set_populations", lambda: sim.set_populations(f0)),
        ("droplets", lambda: sim.droplets([(n / 2, n / 2)])),
        ("check slot", lambda: (sim.set_check(1), sim.step(1), sim.set_check(0))),
        ("adjoint", lambda: sim.adjoint(4, 2, n / 2)),
    ]
    L.lbd_debug_fail_alloc(0)
    sim.set_fields(phi, psi)
    f0 = sim.populations()
    ref = None
    for name, call in calls:
        L.lbd_debug_fail_alloc(1)
        try:
            call()
            failed = False
        except lbd.LbdError as e:
            assert e.code == lbd.LBD_ENOMEM, (name, e)
            failed = True
        L.lbd_debug_fail_alloc(0)
        if failed:
            call()                         # the same call now succeeds
        sim.step(2)
        sim.synchronize()
        d = sim.diagnostics(n / 2, n / 2)
        assert d["status"] == lbd.LBD_OK and d["nonfinite"] == 0, name
    sim.set_fields(phi, psi)
    sim.step(5)
    ref = sim.fields()
    other = lbd.Sim(n, n, precision=lbd.LBD_FP32, tau=0.8, M=0.5)
    other.set_fields(phi, psi)
    other.step(5)
    for a, b in zip(ref, other.fields()):
        assert np.array_equal(a, b)
    sim.close()
    other.close()


def test_3d_create_allocation_failures():
    from paper_1711_10984_gb300 import lbd3
    lbd3.load()
    L = lbd.load()
    for nth in range(1, 12):
        L.lbd_debug_fail_alloc(nth)
        p = lbd3.make_params(lbd.LBD_FP32)
        g = lbd3.lbd3_grid(8, 8, 8)
        h = ctypes.c_void_p()
        rc = L.lbd3_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h))
        if rc == lbd.LBD_OK:
            L.lbd3_destroy(h)
            continue
        assert rc == lbd.LBD_ENOMEM and not h.value, nth
    L.lbd_debug_fail_alloc(0)
