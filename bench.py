#!/usr/bin/env python
"""Throughput benchmark of the coupled LB/FD droplet step on GB300.

Metric: coupled-step MLUPS (million lattice-site updates per second) and the
fraction of the HBM roofline, FP32 (shifted populations) against FP64.

Workload (one GPU): the dilute emulsion, a periodic 2048 x 2048 lattice with 64
seeded droplets of radius 25, seeded surfactant asymmetries and one source disk
per droplet, source and sink active.  A "step" is one coupled time step of the
whole lattice (force, LB collide-and-stream, advection, diffusion, source and
sink); every min(100, K) steps of the step count the diagnostics reduction
(totals, centroid sums, minima, non-finite count: FP64 results) runs as well,
queued on the stream without a host synchronisation (lbd_set_check).  The FP32 state is 369 MB, larger than the 129 MB L2, so no L2
flush is needed between steps.

With --gpus N under torchrun every rank runs its own replica (different seed):
weak scaling, no data-path collective; the timed region is bracketed by
barriers and the maximum over ranks is reported.

--impl reference times the FP64 CPU oracle (the paper's scheme written as plain
C loops) on the host cores, on a 512 x 512 periodic sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled-step MLUPS and % HBM roofline, FP32 vs FP64 on 1 GB300; adjoint/forward cost"
WORKLOAD = ("dilute emulsion: periodic 2048x2048 lattice, 64 seeded droplets R=25, seeded psi "
            "asymmetry, one source disk per droplet, source and sink on")
N_SIDE = 2048
DIAG_EVERY = 100
# Algorithmic HBM bytes per site-step: 9 populations in + 9 out, phi and psi in + out.
BYTES_PER_SITE = {1: 22 * 4, 0: 22 * 8}
# Floating-point operations per site-step of the scheme, counted from the per-site
# arithmetic of each stage done once (no halo recomputation; an FMA counts 2):
# mu_phi and m 61, force 10 + moments 26 + gradient window 26 + BGK/Guo
# collision 92, advection 24, mu*, m* and p* 62, phi/psi updates 58, i.e. 359
# with every gradient scaled by its 1/12; the kernels return 12 grad and fold
# the 1/12 into the constants that use it (12 multiplies fewer, the force's
# body-force add becoming an FMA, m's 1/2 folded into B1): 347.  Nsight
# Compute's FP64 counters on the FP64 step (DADD + DMUL + 2 DFMA) are in the
# FP64 profile summary; the 118 x 128 shape's halo recomputation adds 7 %.
FLOPS_PER_SITE = 347
# FP64 rate of GB300: 1.25 TFLOP/s nominal at the 2070 MHz maximum SM clock,
# scaled to the median SM clock sampled during the run.
FP64_NOMINAL_TFLOPS = 1.25
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_SIDE, help=argparse.SUPPRESS)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(v, dist, device):
    """Maximum of a per-rank scalar over all ranks (v itself without a process group)."""
    if not dist:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(sites_per_rank, world, steps, max_ms):
    """Sites updated by all ranks divided by the slowest rank's time (weak scaling)."""
    return world * sites_per_rank * steps / max_ms / 1e3


def replica_seed(rank):
    return 5 + rank


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def workload(n, seed):
    from paper_1711_10984_gb300 import inputs
    count = 64 if n == N_SIDE else max(1, (n // 256) ** 2)
    return inputs.emulsion(n=n, count=count, seed=seed)


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi samples every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ------------------------------------------------------------------ ours
# Sources of each kernel family, by the launch shape's column count.
KERNEL_SOURCES = {116: ("lbd_vstripe.cu", "lbd_internal.h"),
                  118: ("lbd_stripe.cu", "lbd_internal.h"),
                  246: ("lbd_stripe.cu", "lbd_internal.h")}


def kernel_name(tile, prec):
    t = "float" if prec == 1 else "double"
    if tile[0] == 116:
        return ("vstripe_kernel (FP32, 116-column stripes, row segments of at most %d rows, "
                "as many as fill the resident CTA slots evenly)" % tile[1])
    if tile[0] in (118, 246):
        return "stripe_kernel<%s,%d> (segments of %d rows)" % (t, tile[0] + 10, tile[1])
    return "step_kernel<%s,%d,%d>" % (t, tile[0], tile[1])


def kernel_source_hash(tile):
    """Hash of the sources of the kernel that runs launch shape `tile`."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES.get(tile[0], ("lbd_step.cu", "lbd_internal.h")):
        with open(os.path.join(ROOT, "paper_1711_10984_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(precision, tile):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    if it was taken on the current source of the kernel that runs `tile`;
    else None."""
    name = "step_kernel_%s_emulsion2048.txt" % ("fp32" if precision == 1 else "fp64")
    path = os.path.join(ROOT, "profiles", name)
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_hash:\s*(\w+)", text)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    k = re.search(r"launch_shape:\s*(\d+)x(\d+)", text)
    if not m or not t or m.group(1) != kernel_source_hash(tile):
        return None
    if k and int(k.group(1)) != tile[0]:
        return None
    return float(t.group(1))


def time_precision(torch, lbd, autotune, w, prec, steps, warmup, stream, dev_name, barrier):
    """K timed steps of the whole path: the coupled step every step and the S8
    reduction (lbd_set_check: totals, centroid sums, minima, non-finite count,
    queued on the stream with its result copied to pinned host memory, no host
    synchronisation) every min(100, K) steps of the step count.  Then, outside
    the timed region, K more launches of the step kernel alone, timed with CUDA
    events on the same stream, for the kernel's roofline."""
    sim = lbd.Sim(w["nx"], w["ny"], precision=prec, sources=w["sources"], stream=stream.cuda_stream,
                  **w["params"])
    sim.set_fields(w["phi"], w["psi"])
    tile = autotune.tune(sim, dev_name)
    every = min(DIAG_EVERY, steps)
    sim.set_check(every)
    sim.step(warmup)
    sim.synchronize()
    ref = (w["droplets"][0]["x"], w["droplets"][0]["y"])
    d0 = sim.diagnostics(*ref)
    t0 = sim.t
    ev = lambda: torch.cuda.Event(enable_timing=True)
    barrier()
    e0, e1 = ev(), ev()
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    total_ms = e0.elapsed_time(e1)
    sim.synchronize()  # the checks' verdicts: raises if one found the state broken
    checks = (t0 + steps) // every - t0 // every
    sim.set_check(0)
    k0, k1 = ev(), ev()
    k0.record(stream)
    sim.step(steps)
    k1.record(stream)
    k1.synchronize()
    kernel_ms = k0.elapsed_time(k1)
    d1 = sim.diagnostics(*ref)
    drift = {k: (d1[k] - d0[k]) / abs(d0[k]) for k in ("sum_rho", "sum_phi")}
    sim.close()
    return dict(total_ms=total_ms, kernel_ms=kernel_ms, tile=list(tile),
                launches=steps + 2 * checks, checks=checks, every=every,
                drift=drift, nonfinite=d1["nonfinite"])


def fp64_peak_measured(lbd):
    """The device's FP64 FMA rate in flop/s (lbd_fp64_peak), best of three; None
    if the measurement fails."""
    import ctypes
    best = None
    for _ in range(3):
        v = ctypes.c_double()
        if lbd.load().lbd_fp64_peak(4000, ctypes.byref(v)) == lbd.LBD_OK:
            best = v.value if best is None else max(best, v.value)
    return best


def time_e2e(torch, lbd, autotune, w, steps, stream, dev_name):
    """The same FP32 job through the public API from pinned host memory, in the
    headline's launch shape and diagnostics cadence: upload phi, psi as floats
    (H2D, lbd_set_fields_f32), K steps with the S8 reduction every min(100, K)
    steps (its 9 doubles copied D2H each time), then all five fields read back
    as floats (D2H, lbd_get_fields_f32)."""
    n = w["nx"]
    N = n * n
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    phi_h = pin(np.asarray(w["phi"], dtype=np.float32))
    psi_h = pin(np.asarray(w["psi"], dtype=np.float32))
    outs = [torch.empty(N, dtype=torch.float32).pin_memory().numpy() for _ in range(5)]
    sim = lbd.Sim(n, n, precision=lbd.LBD_FP32, sources=w["sources"], stream=stream.cuda_stream,
                  **w["params"])
    autotune.tune(sim, dev_name)
    every = min(DIAG_EVERY, steps)
    import ctypes
    fp = ctypes.POINTER(ctypes.c_float)
    # one untimed job first: the calls allocate their staging areas on first use
    sim.set_fields_f32(phi_h, psi_h)
    sim.set_check(every)
    sim.step(2)
    sim._check(lbd.load().lbd_get_fields_f32(sim._h, *[o.ctypes.data_as(fp) for o in outs]))
    sim.synchronize()
    times, checks = [], 0
    for rep in range(3):  # three jobs; the median is reported
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        sim.set_fields_f32(phi_h, psi_h)
        t_start = sim.t
        sim.step(steps)
        rc = lbd.load().lbd_get_fields_f32(sim._h, *[o.ctypes.data_as(fp) for o in outs])
        e1.record(stream)
        e1.synchronize()
        wall = time.perf_counter() - t0
        sim._check(rc)
        sim.synchronize()
        checks = (t_start + steps) // every - t_start // every
        times.append(max(e0.elapsed_time(e1), wall * 1e3))
    sim.close()
    ms = sorted(times)[1]
    return dict(ms=ms, h2d=2 * 4 * N, d2h=5 * 4 * N + 9 * 8 * checks, every=every,
                jobs_ms=[round(t, 4) for t in times])


def time_batch(torch, lbd, steps, warmup, count=256):
    """Batched parameter sweep: count independent FP32 single-droplet instances
    (sides 128-384, radii 15-40, B1 and psi amplitude log-uniform), all stepped
    together (persistent launch per step, CUDA-graph replay)."""
    from paper_1711_10984_gb300 import inputs
    ws = inputs.batch_sweep(count=count)
    params = [lbd.make_params(lbd.LBD_FP32, w["sources"], **w["params"]) for w in ws]
    b = lbd.Batch([(w["nx"], w["ny"]) for w in ws], params)
    for k, w in enumerate(ws):
        b.set_fields(k, w["phi"], w["psi"])
    tile = b.autotune(3)
    b.step(max(warmup, 2))
    b.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    b.synchronize()
    el = time.perf_counter() - t0
    sites = sum(w["nx"] * w["ny"] for w in ws)
    b.close()
    return dict(sites=sites, seconds=el, tile=list(tile), count=count,
                mlups=sites * steps / el / 1e6)


def time_adjoint(lbd, steps=4000, ckpt=100):
    """Adjoint workload: 256x256 droplet R=30, FP32 forward, gradient of the
    centroid x-shift w.r.t. psi(0) and B1, checkpoint every 100 steps."""
    from paper_1711_10984_gb300 import inputs
    n = 256
    d = dict(x=n / 2, y=n / 2, R=30.0, psi_mean=0.1, noise=0.01, gx=0.005)
    phi, psi = inputs.droplet_fields(n, n, [d], seed=4)
    kw = dict(inputs.PAPER, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4, t_on=0)
    src = [inputs.default_source(d, n, n)]
    sim = lbd.Sim(n, n, precision=lbd.LBD_FP32, sources=src, **kw)
    sim.set_fields(phi, psi)
    sim.step(10)
    sim.synchronize()
    sim.set_fields(phi, psi)
    sim.t = 0
    t0 = time.perf_counter()
    sim.step(steps)
    sim.synchronize()
    fwd = time.perf_counter() - t0
    sim.set_fields(phi, psi)
    sim.t = 0
    t0 = time.perf_counter()
    L, dpsi, dB1 = sim.adjoint(steps, ckpt, n / 2)
    adj = time.perf_counter() - t0
    sim.close()
    return dict(forward_s=fwd, adjoint_s=adj, ratio=adj / fwd, steps=steps, ckpt_every=ckpt,
                loss=L, dL_dB1=dB1, max_abs_dL_dpsi0=float(np.abs(dpsi).max()))


def time_tracking(lbd, w, reps=20):
    """Per-droplet tracking and the squirmer fit (lbd_droplets + lbd_squirmer) of
    all droplets of the FP32 emulsion: wall clock per call, fields evaluation
    and the synchronising read-back included."""
    n = w["nx"]
    sim = lbd.Sim(n, n, precision=lbd.LBD_FP32, sources=w["sources"], **w["params"])
    sim.set_fields(w["phi"], w["psi"])
    sim.step(10)
    refs = [(d["x"] % n, d["y"] % n) for d in w["droplets"]]
    drops = sim.droplets(refs)
    sim.squirmer(drops)
    t0 = time.perf_counter()
    for _ in range(reps):
        drops = sim.droplets(refs)
    t1 = time.perf_counter()
    for _ in range(reps):
        fit = sim.squirmer(drops)
    t2 = time.perf_counter()
    sim.close()
    return dict(droplets=len(refs), ms_droplets=(t1 - t0) / reps * 1e3,
                ms_squirmer=(t2 - t1) / reps * 1e3,
                points=int(sum(f["points"] for f in fit)))


def time_3d(torch, stream, steps=100, n=256):
    """The 3D (D3Q19) step on a periodic n^3 box with 64 seeded spherical
    droplets (R = 16, a source ball in each, sink on), FP32, CUDA events on the
    launching stream; 5 kernel launches per step."""
    from paper_1711_10984_gb300 import inputs, lbd, lbd3
    lbd3.load()
    w = inputs.emulsion3(n=n)
    sim = lbd3.Sim3(n, n, n, precision=lbd.LBD_FP32, sources=w["sources"],
                    stream=stream.cuda_stream, **w["params"])
    sim.set_fields(w["phi"], w["psi"])
    sim.step(5)
    sim.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    d = sim.diagnostics(*(w["droplets"][0][k] % n for k in ("x", "y", "z")))
    sim.close()
    return dict(n=n, steps=steps, ms_per_step=ms, mlups=n ** 3 / ms / 1e3,
                nonfinite=d["nonfinite"])


def time_small(torch, lbd, autotune, stream, dev_name, steps=500):
    """The small configurations, whose state sits in L2: the 128^2 single
    droplet (FP64) and the 512x256 two-droplet case (FP32 and FP64), each in
    the autotuner's launch shape, CUDA events on the launching stream.  These
    steps are bound by the kernel's latency, not by HBM."""
    from paper_1711_10984_gb300 import inputs
    out = {}
    for name, w, precs in (("single_droplet_128", inputs.single_droplet(), (lbd.LBD_FP64,)),
                           ("two_droplets_512x256", inputs.two_droplets(),
                            (lbd.LBD_FP32, lbd.LBD_FP64))):
        for prec in precs:
            sim = lbd.Sim(w["nx"], w["ny"], precision=prec, sources=w["sources"],
                          stream=stream.cuda_stream, **w["params"])
            sim.set_fields(w["phi"], w["psi"])
            tile = autotune.tune(sim, dev_name)
            sim.step(20)
            sim.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            e1.synchronize()
            us = e0.elapsed_time(e1) / steps * 1e3
            sim.close()
            out["%s_%s" % (name, "fp32" if prec == lbd.LBD_FP32 else "fp64")] = dict(
                sites=w["nx"] * w["ny"], us_per_step=round(us, 2),
                mlups=round(w["nx"] * w["ny"] / us, 1), tile=list(tile))
    return out


def cpu_baseline(w, budget_s=12.0):
    """The FP64 oracle as it stands on the host cores, on the same 2048^2
    workload, for as many whole steps as fit in about budget_s seconds."""
    import oracle
    n = w["nx"]
    p = oracle.Params(n, n, sources=w["sources"], **w["params"])
    s = oracle.State(p, w["phi"], w["psi"])
    t0 = time.perf_counter()
    k = 0
    while True:
        s.step(1)
        k += 1
        el = time.perf_counter() - t0
        if el >= budget_s or k >= 50:
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    out = {"value": n * n * k / el / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": "%d whole steps of the %dx%d workload (FP64, C oracle, OpenMP rows)"
                     % (k, n, n)}
    # the same oracle on one core, on a 512 x 512 window of the workload
    try:
        import ctypes
        gomp = ctypes.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(1)
        m = 512
        p1 = oracle.Params(m, m, sources=[src for src in w["sources"] if src[0] < m and src[1] < m],
                           **w["params"])
        s1 = oracle.State(p1, w["phi"][:m, :m], w["psi"][:m, :m])
        t0 = time.perf_counter()
        k1 = 0
        while True:
            s1.step(1)
            k1 += 1
            el1 = time.perf_counter() - t0
            if el1 >= budget_s / 2 or k1 >= 200:
                break
        out["one_core"] = {"value": m * m * k1 / el1 / 1e6, "unit": "MLUPS", "cores": 1,
                           "sample": "%d whole steps of a %dx%d periodic window" % (k1, m, m)}
    except OSError:
        pass
    finally:
        try:
            gomp.omp_set_num_threads(cores)
        except NameError:
            pass
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_1711_10984_gb300 import autotune, lbd
    lbd.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    barrier = (lambda: dist.barrier()) if dist else (lambda: None)
    dev_name = torch.cuda.get_device_name(local)
    w = workload(args.n, seed=replica_seed(rank))
    N = args.n * args.n
    stream = torch.cuda.Stream()
    clocks = Clocks(local)
    clocks.start()
    r32 = time_precision(torch, lbd, autotune, w, lbd.LBD_FP32, args.steps, args.warmup, stream,
                         dev_name, barrier)
    r64 = time_precision(torch, lbd, autotune, w, lbd.LBD_FP64, args.steps, args.warmup, stream,
                         dev_name, barrier)
    clk = clocks.stop()
    fp64_rate = fp64_peak_measured(lbd)
    e2e = time_e2e(torch, lbd, autotune, w, args.steps, stream, dev_name)
    batch = time_batch(torch, lbd, min(args.steps, 500), args.warmup)
    # the adjoint workload at its own size, whatever --steps is
    adj = time_adjoint(lbd, steps=4000, ckpt=100) if rank == 0 else None
    # walls (bounce-back plates): the same emulsion between plates, and the
    # channel of Section 4 (512 x 256, one droplet R = 32, tau = 0.6)
    from paper_1711_10984_gb300 import inputs
    w_pl = dict(w, params=dict(w["params"], flags=lbd.LBD_WALLS))
    nw = min(args.steps, 500)
    rw = time_precision(torch, lbd, autotune, w_pl, lbd.LBD_FP32, nw, args.warmup, stream,
                        dev_name, barrier)
    wc = inputs.channel()
    rc = time_precision(torch, lbd, autotune, wc, lbd.LBD_FP32, nw, args.warmup, stream,
                        dev_name, barrier)
    trk = time_tracking(lbd, w) if rank == 0 else None
    r3 = time_3d(torch, stream, steps=min(args.steps, 100))
    small = time_small(torch, lbd, autotune, stream, dev_name, steps=min(args.steps, 500))

    maxr = lambda v: max_over_ranks(v, dist, "cuda")

    t32, t64, te = maxr(r32["total_ms"]), maxr(r64["total_ms"]), maxr(e2e["ms"])
    k32, k64 = maxr(r32["kernel_ms"]), maxr(r64["kernel_ms"])
    tw, kw, tc = maxr(rw["total_ms"]), maxr(rw["kernel_ms"]), maxr(rc["total_ms"])
    cpu = cpu_baseline(w) if (rank == 0 and world == 1) else None
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    hbm, src = peaks()
    mlups32 = whole_job_mlups(N, world, args.steps, t32)
    mlups64 = whole_job_mlups(N, world, args.steps, t64)
    ach32 = BYTES_PER_SITE[1] * N / (k32 / args.steps * 1e-3) / 1e9
    ach64_gbs = BYTES_PER_SITE[0] * N / (k64 / args.steps * 1e-3) / 1e9
    flops64 = FLOPS_PER_SITE * N / (k64 / args.steps * 1e-3) / 1e12
    mhz = clk.get("sm_mhz") or SM_MAX_MHZ
    if fp64_rate:
        fp64_peak, fp64_src = fp64_rate / 1e12, (
            "measured: lbd_fp64_peak (independent FP64 FMAs on every SM, CUDA events)")
    else:
        fp64_peak, fp64_src = FP64_NOMINAL_TFLOPS * mhz / SM_MAX_MHZ, (
            "nominal 1.25 TFLOP/s at 2070 MHz x median SM clock (measurement failed)")
    out = {
        "metric": METRIC, "value": round(mlups32, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t32 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sites_per_gpu": N, "precision": "FP32 shifted populations",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "state 369 MB > 129 MB L2, no flush", "tile": r32["tile"],
                   "diagnostics_every": r32["every"], "diagnostics_in_timed_region": r32["checks"]},
        "roofline": {"bound": "hbm", "achieved": round(ach32, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(ach32 / hbm, 4), "traffic": ncu_traffic(1, r32["tile"]),
                     "peak_source": src, "kernel": kernel_name(r32["tile"], 1),
                     "timing": "CUDA events around %d back-to-back launches on the launching "
                               "stream" % args.steps,
                     "bytes_per_site": BYTES_PER_SITE[1]},
        "fp64": {"value": round(mlups64, 1), "unit": "MLUPS", "ms_per_step": t64 / args.steps,
                 "dtype": "f64", "tile": r64["tile"],
                 "roofline": {"bound": "alu", "achieved": round(flops64, 4),
                              "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                              "frac": round(flops64 / fp64_peak, 4),
                              "peak_source": fp64_src,
                              "flops_per_site": FLOPS_PER_SITE,
                              "hbm_gbs_achieved": round(ach64_gbs, 1),
                              "hbm_frac": round(ach64_gbs / hbm, 4),
                              "traffic": ncu_traffic(0, r64["tile"]),
                              "kernel": kernel_name(r64["tile"], 0),
                              "nominal_tflops": FP64_NOMINAL_TFLOPS},
                 "drift": r64["drift"]},
        "fp32_over_fp64_speedup": round(t64 / t32, 2),
        "fp32_drift": r32["drift"],
        "adjoint_forward_cost": adj,
        "tracking": trk,
        "small_configs": dict(small, note="state in L2; latency-bound steps, no roofline"),
        "three_d": {"workload": "D3Q19 coupled step, periodic 256^3 box, 64 seeded spherical "
                                "droplets R=16 with a source ball each, sink on, FP32",
                    "value": round(world * r3["mlups"], 1), "unit": "MLUPS",
                    "ms_per_step": r3["ms_per_step"], "steps": r3["steps"],
                    "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm,
                                 "bytes_per_site": 168,
                                 "achieved": round(r3["mlups"] * 1e6 * 168 / 1e9, 1),
                                 "frac": round(r3["mlups"] * 1e6 * 168 / 1e9 / hbm, 4)},
                    "nonfinite": r3["nonfinite"]},
        "walls": {"workload": "the same 2048x2048 emulsion between bounce-back plates "
                              "(LBD_WALLS), FP32",
                  "value": round(whole_job_mlups(N, world, nw, tw), 1),
                  "unit": "MLUPS", "steps": nw, "tile": rw["tile"],
                  "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm,
                               "achieved": round(BYTES_PER_SITE[1] * N / (kw / nw * 1e-3) / 1e9, 1),
                               "frac": round(BYTES_PER_SITE[1] * N / (kw / nw * 1e-3) / 1e9 / hbm,
                                             4)},
                  "channel": {"workload": "Section 4 channel: 512x256 between plates, one droplet "
                                          "R=32, tau=0.6, B1=-0.05, source and sink on, FP32",
                              "value": round(whole_job_mlups(wc["nx"] * wc["ny"], world, nw, tc), 1),
                              "unit": "MLUPS", "tile": rc["tile"], "ms_per_step": tc / nw}},
        "batch": {"workload": "256 FP32 single-droplet instances, sides 128-384, radii 15-40, "
                              "B1 and psi amplitude log-uniform, source and sink on",
                  "value": round(world * batch["mlups"], 1), "unit": "MLUPS",
                  "sites": batch["sites"], "steps": min(args.steps, 500), "tile": batch["tile"],
                  "hbm_frac": round(batch["mlups"] * 1e6 * BYTES_PER_SITE[1] / 1e9 / hbm, 4),
                  "timing": "wall clock around lbd_batch_step + synchronize (graph replays)"},
        "e2e": {"value": round(world * N * args.steps / te / 1e3, 1), "unit": "MLUPS",
                "h2d_bytes_per_step": e2e["h2d"] / args.steps,
                "d2h_bytes_per_step": e2e["d2h"] / args.steps,
                "what": "one job of K=%d steps through the C ABI: lbd_set_fields_f32 from "
                        "pinned host float phi/psi, lbd_step(K) with the S8 reduction every %d "
                        "steps (its 9 doubles copied to pinned host memory), lbd_get_fields_f32 "
                        "of rho, u, phi, psi to pinned host floats; median of 3 such jobs, after "
                        "one untimed job" % (args.steps, e2e["every"]),
                "jobs_ms": e2e["jobs_ms"]},
        "clocks": clk,
        "gpu_launches": r32["launches"],
    }
    if cpu:
        out["cpu_baseline"] = cpu
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ reference
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    n_full = args.n
    w = workload(n_full, seed=5)
    ns = min(512, n_full)
    # periodic 512 x 512 sample: the window's own droplets and sources
    phi = np.ascontiguousarray(w["phi"][:ns, :ns])
    psi = np.ascontiguousarray(w["psi"][:ns, :ns])
    srcs = [s for s in w["sources"] if s[0] < ns and s[1] < ns]
    p = oracle.Params(ns, ns, sources=srcs, **w["params"])
    s = oracle.State(p, phi, psi)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    el = time.perf_counter() - t0
    v = ns * ns * args.steps / el / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    sample = "%dx%d periodic window of the workload per step (FP64 C oracle)" % (ns, ns)
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        run_reference(args)
    else:
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
        run_ours(args)


if __name__ == "__main__":
    main()
