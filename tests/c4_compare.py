"""C4 precision sweep, oracle side (test infrastructure, runs on the host).

`bench.py --sweep STEPS --sweep-n N --sweep-out DIR` runs the C4 cylinder on
the GPU in FP32 (float atomics), FP32 + int64 fixed point (unit 1 and
normalised units) and FP64, and writes each mode's fields by particle id to
DIR.  This script runs the FP64 oracle on the same initial state for the same
number of steps and reports, per mode, the relative L1 and L-infinity errors
of rho, |V|, P and e against it over the particle ids the GPU side wrote
(every 8th), with the bit-reproducibility flags it recorded (all particles):

    python tests/c4_compare.py DIR --steps 1000 --n 1024 [--json OUT]

The oracle runs --steps steps; its final time is what the GPU side should be
given as --sweep-t-end (CFL steps depend on the largest particle speed, so
equal step counts are not equal times).  Each mode's fields are compared at
that time.

Particles whose position differs from the oracle's by more than one cell
(a recycling decision taken one step apart) are left out and counted.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
import bench  # noqa: E402


def errors(g: dict, R: dict, h: float) -> dict:
    far = np.abs(g["X"] - R["X"]).max(axis=0) > h
    ok = ~far
    err = {"excluded_far": int(far.sum())}
    for f in ("RHO", "P", "E"):
        d = np.abs(g[f][ok] - R[f][ok])
        err[f] = {"rel_l1": float(d.sum() / np.abs(R[f][ok]).sum()),
                  "rel_linf": float(d.max() / np.abs(R[f][ok]).max())}
    vm = np.sqrt((R["V"][:, ok] ** 2).sum(axis=0))
    dv = np.sqrt(((g["V"][:, ok] - R["V"][:, ok]) ** 2).sum(axis=0))
    err["V"] = {"rel_l1": float(dv.sum() / vm.sum()), "rel_linf": float(dv.max() / vm.max())}
    return err


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("dir")
    ap.add_argument("--steps", type=int, required=True)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--json", default=None)
    ap.add_argument("--oracle-cache", default=None,
                    help="npz file with the oracle's fields: read if it exists, else written")
    a = ap.parse_args()
    base = bench.c4_problem(a.n)
    if a.oracle_cache and os.path.exists(a.oracle_cache):
        z = np.load(a.oracle_cache)
        R = {f: z[f] for f in ("RHO", "P", "E", "V", "X")}
        clock, t_or = z["clock"], float(z["seconds"])
    else:
        ref = O.OracleSim(base.cfg)
        ref.add_particles(base.x, base.v, base.mass, base.rho, base.e)
        ref.set_obstacle_mask(base.mask, base.normals)
        t0 = time.perf_counter()
        ref.step(a.steps)
        t_or = time.perf_counter() - t0
        io = np.argsort(ref.read("ID"))
        R = {f: ref.read(f)[..., io] for f in ("RHO", "P", "E", "V", "X")}
        clock = ref.read("CLOCK")
        if a.oracle_cache:
            np.savez(a.oracle_cache, clock=clock, seconds=t_or, **R)
    if int(clock[2]) != a.steps:
        raise SystemExit(f"oracle ran {int(clock[2])} steps, not {a.steps}")
    out = {"workload": f"cylinder {a.n}x{a.n // 2}, {base.n_particles} particles, {a.steps} steps",
           "oracle": {"seconds": t_or, "t": float(clock[0]), "steps": int(clock[2])}, "modes": {}}
    sweep = {}
    sj = os.path.join(a.dir, "c4_sweep.json")
    if os.path.exists(sj):
        sweep = json.load(open(sj)).get("sweep", {}).get("modes", {})
    for name, _, _ in bench.c4_modes(base):
        f = os.path.join(a.dir, f"c4_{name}.npz")
        if not os.path.exists(f):
            continue
        z = np.load(f)
        k = int(z["sample"])
        g = {f: z[f].astype(np.float64) for f in ("RHO", "P", "E", "V", "X")}
        Rk = {f: a[..., ::k] for f, a in R.items()}
        if abs(float(z["clock"][0]) - float(clock[0])) > 1e-12 * float(clock[0]):
            print(f"warning: {name} is at t = {float(z['clock'][0])!r}, the oracle at {float(clock[0])!r}")
        m = {"errors": errors(g, Rk, base.cfg["h"]), "t": float(z["clock"][0]), "steps": int(z["clock"][2]),
             "particles_compared": int(g["RHO"].shape[0]), "every_nth_id": k}
        if name in sweep:
            m["bit_reproducible"] = sweep[name]["bit_reproducible"]
        out["modes"][name] = m
    s = json.dumps(out, indent=1)
    print(s)
    if a.json:
        with open(a.json, "w") as fh:
            fh.write(s + "\n")


if __name__ == "__main__":
    main()
