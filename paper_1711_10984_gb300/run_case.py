"""Run one of the seeded droplet workloads from the command line.

    python -m paper_1711_10984_gb300.run_case --workload emulsion --n 2048 \
        --precision fp32 --steps 10 [--tile 32x16] [--check-every 20]
    python -m paper_1711_10984_gb300.run_case --workload emulsion3 --n 128 \
        --droplets 8 --radius 12 --steps 7          (the 3D step on an n^3 box)
    python -m paper_1711_10984_gb300.run_case --workload adjoint --n 256 \
        --steps 200 --ckpt 100                      (FP32 forward + hand adjoint)

Prints the final diagnostics.  Used as the profiling target of the ncu
summaries under profiles/.
"""
import argparse
import json

from . import inputs, lbd


def make(workload, n):
    if workload == "emulsion":
        return inputs.emulsion(n=n, count=64 if n == 2048 else max(1, (n // 256) ** 2), seed=5)
    if workload == "single":
        return inputs.single_droplet(n=n)
    if workload == "two":
        return inputs.two_droplets()
    raise ValueError(workload)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="emulsion",
                    choices=["emulsion", "single", "two", "emulsion3", "adjoint"])
    ap.add_argument("--droplets", type=int, default=64, help="emulsion3: droplet count")
    ap.add_argument("--radius", type=float, default=16.0, help="emulsion3: droplet radius")
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--tile", default=None)
    ap.add_argument("--ckpt", type=int, default=100, help="adjoint: checkpoint interval")
    ap.add_argument("--check-every", type=int, default=0,
                    help="run-time checks (the S8 reduction) every k steps (lbd_set_check)")
    a = ap.parse_args(argv)
    prec = lbd.LBD_FP32 if a.precision == "fp32" else lbd.LBD_FP64
    if a.workload == "emulsion3":
        from . import lbd3
        lbd3.load()
        w = inputs.emulsion3(n=a.n, count=a.droplets, R=a.radius)
        sim = lbd3.Sim3(a.n, a.n, a.n, precision=prec, sources=w["sources"], **w["params"])
        sim.set_fields(w["phi"], w["psi"])
        sim.step(a.steps)
        d0 = w["droplets"][0]
        print(json.dumps(sim.diagnostics(d0["x"] % a.n, d0["y"] % a.n, d0["z"] % a.n)))
        sim.close()
        return
    if a.workload == "adjoint":
        # one droplet R = 30 on n x n, source on; gradient of the centroid x-shift
        n = a.n
        d = dict(x=n / 2, y=n / 2, R=30.0, psi_mean=0.1, noise=0.01, gx=0.005)
        phi, psi = inputs.droplet_fields(n, n, [d], seed=4)
        kw = dict(inputs.PAPER, gamma=1.5e-3, c0=0.09, A0=1.5e-10, A_max=1e-4, t_on=0)
        sim = lbd.Sim(n, n, precision=prec, sources=[inputs.default_source(d, n, n)], **kw)
        sim.set_fields(phi, psi)
        L, _, dB1 = sim.adjoint(a.steps, a.ckpt, n / 2, want_dpsi=False)
        print(json.dumps(dict(loss=L, dL_dB1=dB1)))
        sim.close()
        return
    w = make(a.workload, a.n)
    sim = lbd.Sim(w["nx"], w["ny"], precision=prec, sources=w["sources"], **w["params"])
    if a.tile:
        sim.set_tile(*[int(v) for v in a.tile.split("x")])
    sim.set_fields(w["phi"], w["psi"])
    sim.set_check(a.check_every)
    sim.step(a.steps)
    sim.synchronize()
    d = sim.diagnostics(w["droplets"][0]["x"] % w["nx"], w["droplets"][0]["y"] % w["ny"])
    print(json.dumps(d))
    sim.close()


if __name__ == "__main__":
    main()
