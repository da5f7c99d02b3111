"""Run one of the seeded droplet workloads from the command line.

    python -m paper_1711_10984_gb300.run_case --workload emulsion --n 2048 \
        --precision fp32 --steps 10 [--tile 32x16]

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
    ap.add_argument("--workload", default="emulsion", choices=["emulsion", "single", "two"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--tile", default=None)
    a = ap.parse_args(argv)
    w = make(a.workload, a.n)
    prec = lbd.LBD_FP32 if a.precision == "fp32" else lbd.LBD_FP64
    sim = lbd.Sim(w["nx"], w["ny"], precision=prec, sources=w["sources"], **w["params"])
    if a.tile:
        sim.set_tile(*[int(v) for v in a.tile.split("x")])
    sim.set_fields(w["phi"], w["psi"])
    sim.step(a.steps)
    d = sim.diagnostics(w["droplets"][0]["x"] % w["nx"], w["droplets"][0]["y"] % w["ny"])
    print(json.dumps(d))
    sim.close()


if __name__ == "__main__":
    main()
