#!/usr/bin/env python
"""Benchmark of the MPM hot path on one B300 (or N, as independent replicas).

Workload (default): 3D blast wave, 256^3 cells on the unit cube, 2x2x2
particles per cell (134,217,728 particles), quadratic B-splines, FP32, slip
walls, CFL 0.3 -- the configuration on which the HBM-roofline target is set.

A step is one pass of the whole hot path: P2G, grid update + G2P + P2G,
G2PD + particle update + move, time advance and the stable re-order.  The
metric is particle-steps per second.  Inputs are resident in HBM when the
timed region starts (particle state ~13 GB, far larger than the 126 MB L2,
so no L2 flush is needed between steps).  Per-phase device times come from
CUDA events that the library records on its own stream; the clocks are
sampled with nvidia-smi during the timed region.

python bench.py [--gpus N] [--steps K] [--warmup W] [--config blast|cylinder]
python bench.py --impl reference ...   (the FP64 CPU oracle on host cores)
Under torchrun each rank runs its own independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import glob
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6400.0
NOMINAL_HBM = 7700.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--config", default="blast", choices=["blast", "cylinder", "cylinder_paper"],
                    help="cylinder: the 1024x512 C2 set-up; cylinder_paper: the paper's own cylinder geometry "
                         "([0,4]x[0,2], r = 0.25 at (0.6, 1), CFL 1/2; --n x cells)")
    ap.add_argument("--n", type=int, default=0, help="override the grid size (cells per axis / x cells)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp32_coloured", "fp32_fixed64", "fp64"])
    ap.add_argument("--degree", type=int, default=2, choices=[1, 2], help="basis: 1 = Q1, 2 = quadratic B-spline")
    ap.add_argument("--ppa", type=int, default=2, help="particles per cell along each axis")
    ap.add_argument("--tile", default="",
                    help="tile edges in spans, e.g. 8x8x8 (default: 8x8x8 for the blast, the library's for the "
                         "cylinders)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serve", type=int, default=0,
                    help="also run the serving stream with this many requests (batched vs one at a time)")
    ap.add_argument("--serve-steps", type=int, default=500)
    ap.add_argument("--saturated", action="store_true", help="serving: all requests arrive at t=0")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--sweep", type=int, default=0,
                    help="C4 precision sweep on the cylinder with this many steps (0: skip)")
    ap.add_argument("--sweep-n", type=int, default=1024, help="cylinder x cells for the sweep")
    ap.add_argument("--sweep-out", default="c4_fields", help="directory for the sweep's fields")
    ap.add_argument("--sweep-t-end", type=float, default=0.0,
                    help="run every mode to this simulated time instead of a step count (the time the FP64 oracle "
                         "reaches in --sweep steps): CFL steps depend on the largest particle speed, so equal step "
                         "counts are not equal times")
    return ap.parse_args()


# Tile edges (spans) of the GPU kernels per workload, timed on B300: for the
# 256^3 blast 8x8x8 10.43, 16x4x8 10.59, 16x8x4 (the library default) 10.68,
# 8x16x4 10.73, 4x8x16 10.73, 32x4x4 12.38, 16x8x8 13.34 ms per step; the
# 1024x512 cylinder keeps the library's 32x8 (16x16, 64x4, 32x4: +1 to +6%).
DEFAULT_TILE = {"blast": [8, 8, 8]}


def tile_of(args):
    if args.tile:
        t = [int(v) for v in args.tile.split("x")]
        return t + [0] * (3 - len(t))
    return DEFAULT_TILE.get(args.config, [0, 0, 0])


def workload(args):
    """The workload's description, from the arguments alone (both arms)."""
    basis = "quadratic B-spline" if args.degree == 2 else "Q1"
    tile = tile_of(args)
    if args.config == "blast":
        n = args.n or 256
        ppc = args.ppa ** 3
        return {"workload": f"3D blast wave {n}^3 cells, {ppc} ppc, {basis}, {args.precision}",
                "cells": [n, n, n], "ppc": ppc, "degree": args.degree, "precision": args.precision,
                "tile": tile if any(tile) else "library default"}
    nx = args.n or (1024 if args.config == "cylinder" else 1414)
    ppc = args.ppa ** 2
    where = "" if args.config == "cylinder" else " on [0,4]x[0,2], r = 0.25, CFL 1/2"
    return {"workload": f"2D Mach-3 cylinder {nx}x{nx // 2} cells{where}, {ppc} ppc, {basis}, {args.precision}",
            "cells": [nx, nx // 2], "ppc": ppc, "degree": args.degree, "precision": args.precision,
            "tile": tile if any(tile) else "library default"}


def problem(args):
    from paper_2404_17057_b300 import inputs as I
    cfg = workload(args)
    if args.config == "blast":
        n = cfg["cells"][0]
        p = I.blast(n=n, ppa=args.ppa, degree=args.degree, precision=args.precision, tile=tile_of(args))
        cfg["l2"] = "inputs larger than L2 (no flush)"
    else:
        nx, ny = cfg["cells"]
        geo = {} if args.config == "cylinder" else {"lx": 4.0, "center": (0.6, 1.0), "radius": 0.25, "cfl": 0.5}
        p = I.cylinder(nx=nx, ny=ny, ppa=args.ppa, degree=args.degree, precision=args.precision, tile=tile_of(args),
                       **geo)
        cfg["l2"] = ("inputs larger than L2 (no flush)" if p.n_particles * 40 > 126e6
                     else "particle state partly L2-resident")
    cfg["particles"] = p.n_particles
    return p, cfg


def algorithmic_bytes(dim, s, n_p, n_n, g=None):
    """Bytes each kernel must move at minimum (one read/write per word); s is
    the particle word size, g the grid word size (8 for the int64 grid of the
    fixed-point mode; default s).
    K1 P2G: particles read x,v,M,rho,e,q (2d+4 words); nodes written m,mv,f (2d+1).
    K2 grid+G2P+P2G: particles read x,v,M (2d+1), write v (d); nodes read m,f (1+d), write mv2 (d).
    K3 G2PD+update: particles read x,rho,e,q (d+3), write x,rho,e,q (d+3) and a 4-byte key;
                    nodes read m,mv,f,mv2 (1+3d).
    zeroing: nodes written (1+3d)."""
    g = s if g is None else g
    k1 = n_p * (2 * dim + 4) * s + n_n * (2 * dim + 1) * g
    k2 = n_p * (3 * dim + 1) * s + n_n * (1 + 2 * dim) * g
    k3 = n_p * ((2 * dim + 6) * s + 4) + n_n * (1 + 3 * dim) * g
    zero = n_n * (1 + 3 * dim) * g
    return {"p2g": k1 + zero, "grid_g2p": k2, "g2pd": k3}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: let its first sample arrive,
            # then keep only samples taken from the start of the timed region
            t0 = time.perf_counter()
            while not self.rows and time.perf_counter() - t0 < 5.0:
                time.sleep(0.01)
            self.first = len(self.rows)
        except Exception:
            self.proc = None

    def mark(self):
        """The timed region starts now."""
        self.first = len(self.rows)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.rows = self.rows[getattr(self, "first", 0):]
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(self.rows)}
        try:
            sm = [float(r[1]) for r in self.rows if len(r) >= 9]
            if sm:
                out["sm_mhz"] = float(np.median(sm))
                out["sm_max_mhz"] = float(self.rows[0][2])
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for i, nme in enumerate(names):
                if any(len(r) >= 9 and r[5 + i].lower() == "active" for r in self.rows):
                    out["reasons"].append(nme)
        except Exception:
            pass
        return out


# DRAM bytes per particle of the step kernels, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch each) of the
# 128^3 blast, FP32, degree 2, 8x8x8 tiles, second step, divided by its
# 16,777,216 particles.  Traffic grows with the particle count (same tiles,
# same ppc), so a full 256^3 launch moves 8x those bytes.  Valid only for the
# kernel sources with this digest.
MEASURED_TRAFFIC = {
    "sources": "8928d4484630a990",
    "config": ("blast", 3, 2, "fp32", 2, (8, 8, 8)),
    "bytes_per_particle": {"p2g": 47.70, "grid_g2p": 44.11, "g2pd": 54.05, "reorder": 0.044},
}


def sources_digest() -> str:
    """Digest of the kernel sources' code: comments and blank lines are
    dropped, so that a comment edit keeps the measured counters valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2404_17057_b300", "csrc", "*.cu*"))):
        with open(f, encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(os.path.basename(f).encode() + b"\0" + code.encode())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, config: str, dim: int, degree: int, precision: str, ppa: int, n_p: int,
                     tile=(0, 0, 0)):
    """DRAM bytes of one launch of `kernel`, or None when the counters were
    taken on other kernel sources or another kind of workload."""
    t = MEASURED_TRAFFIC
    if t["config"] != (config, dim, degree, precision, ppa, tuple(tile)) or sources_digest() != t["sources"]:
        return None
    return t["bytes_per_particle"][kernel] * n_p


def peaks():
    try:
        d = json.load(open(PEAKS))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def cpu_baseline(args, cfg_meta, seconds_budget=20.0):
    """The FP64 oracle as it stands, on the host, on a bounded sample of the
    same workload (a smaller grid of the same problem, a few steps)."""
    from oracle import oracle as O
    from paper_2404_17057_b300 import inputs as I
    if args.config == "blast":
        n = 32
        p = I.blast(n=n, ppa=args.ppa, degree=args.degree, precision="fp64")
        sample = (f"blast {n}^3 cells ({args.ppa ** 3} ppc, {p.n_particles} particles), same ppc/basis, "
                  f"FP64 oracle")
    else:
        n = 128
        geo = {} if args.config == "cylinder" else {"lx": 4.0, "center": (0.6, 1.0), "radius": 0.25, "cfl": 0.5}
        p = I.cylinder(nx=n, ny=n // 2, ppa=args.ppa, degree=args.degree, precision="fp64", **geo)
        sample = (f"cylinder {n}x{n // 2} cells ({args.ppa ** 2} ppc, {p.n_particles} particles), same "
                  f"ppc/basis, FP64 oracle")
    s = O.OracleSim(p.cfg)
    s.add_particles(p.x, p.v, p.mass, p.rho, p.e)
    if p.mask is not None:
        s.set_obstacle_mask(p.mask, p.normals)
    s.step(1)
    steps, t0 = 0, time.perf_counter()
    while True:
        s.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > seconds_budget or steps >= 200:
            break
    rate = p.n_particles * steps / el
    return {"value": rate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample}, {steps} steps in {el:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    meta = workload(args)
    cb = cpu_baseline(args, meta, seconds_budget=max(5.0, min(60.0, 3.0 * (args.steps + args.warmup))))
    line = {"impl": "reference", "metric": "particle-steps/s", "value": cb["value"], "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": meta, "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serving(args):
    """C5: continuous batching vs one-at-a-time plain solves on the same stream.
    Tile shapes are tuned once per problem class before either arm is timed
    and both arms use them."""
    from paper_2404_17057_b300 import inputs as I, serve as S, tune as T
    reqs = I.serving_stream(count=args.serve, seed=5, steps=args.serve_steps)
    rt = not args.saturated
    tuner = T.TileTuner()
    t0 = time.perf_counter()
    seen = set()
    for r in reqs:
        if (r["kind"], r["side"]) not in seen:
            seen.add((r["kind"], r["side"]))
            tuner.tile_for(I.request_problem(r))
    tune_s = time.perf_counter() - t0
    _, batched = S.Server(tuner=tuner).run(reqs, realtime=rt)
    _, single = S.run_sequential(reqs, realtime=rt, tuner=tuner)
    return {"requests": len(reqs), "steps_each": args.serve_steps, "arrivals": "all at t=0" if args.saturated
            else "Poisson 50/s", "precision": "fp32_fixed64", "batched": batched, "one_at_a_time": single,
            "speedup_solves_per_s": batched["solves_per_s"] / single["solves_per_s"],
            "tiles": {"classes": len(tuner.table), "tuning_seconds": tune_s, "chosen": tuner.table}}


def c4_modes(base):
    """The C4 precision modes: name, precision, fixed-point units (mass,
    momentum, force).  Normalised units: mean particle mass, that times the
    free-stream speed plus sound speed, and that over 1e-4 (about the first
    CFL step)."""
    um = float(base.mass.mean())
    umom = um * (3.0 + 1.0)
    return [("fp32", "fp32", None), ("fp32_fixed64_unit1", "fp32_fixed64", [1.0, 1.0, 1.0]),
            ("fp32_fixed64_normalised", "fp32_fixed64", [um, umom, umom / 1e-4]), ("fp64", "fp64", None)]


def c4_problem(n):
    """The C4 cylinder (C2 geometry, n x n/2 cells, 2x2 stratified ppc, seed 1)
    with its initial state rounded to binary32, so that every mode and the
    FP64 oracle start from the same values."""
    from paper_2404_17057_b300 import inputs as I
    base = I.cylinder(nx=n, ny=n // 2, precision="fp64")
    for k in ("x", "v", "mass", "rho", "e"):
        setattr(base, k, getattr(base, k).astype(np.float32).astype(np.float64))
    return base


C4_SAMPLE = 8   # the fields of every 8th particle id are written


def sweep(args):
    """C4 on the GPU: the cylinder in FP32 (float atomics), FP32 + int64 fixed
    point (unit 1 and normalised units) and FP64, each run twice for
    `--sweep` steps.  Reports whether the two runs agree bit for bit (all
    particles) and writes each mode's fields of every C4_SAMPLE-th particle
    id, in the storage precision, to `--sweep-out`/c4_<mode>.npz.  The
    comparison with the FP64 oracle is tests/c4_compare.py."""
    from paper_2404_17057_b300 import inputs as I, mpm as M
    n = args.sweep_n
    base = c4_problem(n)
    os.makedirs(args.sweep_out, exist_ok=True)
    span = f"to t = {args.sweep_t_end!r}" if args.sweep_t_end > 0 else f"{args.sweep} steps"
    out = {"workload": f"cylinder {n}x{n // 2}, {base.n_particles} particles, {span}",
           "dir": args.sweep_out, "modes": {}}
    for name, prec, unit in c4_modes(base):
        runs = []
        for _ in range(2):
            cfg = dict(base.cfg, precision=prec)
            if unit:
                cfg["fixed_unit"] = unit
            p = I.Problem("c4", cfg, base.x, base.v, base.mass, base.rho, base.e, base.mask, base.normals)
            g = M.Simulation.from_problem(p)
            t0 = time.perf_counter()
            if args.sweep_t_end > 0:
                g.step(100 * args.sweep, t_end=args.sweep_t_end)
            else:
                g.step(args.sweep)
            sec = time.perf_counter() - t0
            ig = np.argsort(g.read("ID"))
            runs.append({f: g.read(f)[..., ig] for f in ("RHO", "P", "E", "V", "X")})
            clock = g.read("CLOCK")
            g.close()
        same = all(np.array_equal(runs[0][f], runs[1][f]) for f in runs[0])
        dt = np.float64 if prec == "fp64" else np.float32
        np.savez(os.path.join(args.sweep_out, f"c4_{name}.npz"), clock=clock, sample=C4_SAMPLE,
                 **{f: a[..., ::C4_SAMPLE].astype(dt) for f, a in runs[0].items()})
        out["modes"][name] = {"bit_reproducible": bool(same), "seconds": sec, "t": float(clock[0]),
                              "steps": int(clock[2])}
    return out


def max_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (the job ends when its last rank does)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_p: int, steps: int, world: int, ms: float) -> float:
    """Whole-job particle-steps/s: every rank advances its own replica of
    n_p particles for `steps` steps (weak scaling); ms is the slowest rank's
    time."""
    return n_p * steps * world / (ms / 1e3)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        import torch  # noqa: F401  (device memory through the binding)
        print(json.dumps({"metric": "precision sweep", "sweep": sweep(args)}), flush=True)
        return
    import torch
    from paper_2404_17057_b300 import build as B, mpm as M

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    B.build()
    p, meta = problem(args)
    n_p = p.n_particles

    sim = M.Simulation.from_problem(p)
    st = torch.cuda.ExternalStream(sim.stream)
    sim.step(args.warmup)
    t_sim0 = float(sim.read("CLOCK")[0])
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    # the timed region: the production path (one CUDA graph per step)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    sim.step_async(args.steps)
    e1.record(st)
    sim.sync()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    t_sim1 = float(sim.read("CLOCK")[0])
    if dist:
        dist.barrier()
    # per-phase device times: the same steps again with events between phases
    prof_steps = max(1, min(args.steps, 10))
    sim.profile(True)
    sim.profile_read(reset=True)
    sim.step(prof_steps)
    phase_ms, counts = sim.profile_read(reset=True)
    sim.profile(False)
    sizes = sim.sizes()
    n_n = sizes["nodes"]
    value = job_value(n_p, args.steps, world, ms)

    dim = p.cfg["dim"]
    s = 8 if args.precision == "fp64" else 4
    alg = algorithmic_bytes(dim, s, n_p, n_n, 8 if args.precision in ("fp64", "fp32_fixed64") else 4)
    names = ["p2g", "grid_g2p", "g2pd"]
    per_launch_ms = {nme: phase_ms[i] / prof_steps for i, nme in enumerate(names)}
    dom = max(names, key=lambda k: per_launch_ms[k])
    hbm, which = peaks()
    ach = alg[dom] / (per_launch_ms[dom] / 1e3) / 1e9
    k123_ms = sum(per_launch_ms.values())
    k123_gbs = sum(alg.values()) / (k123_ms / 1e3) / 1e9
    launches_per_step = int(counts[0] + counts[1] + counts[2] + counts[3] + counts[4] + 1)

    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = end_to_end(M, p, args)
    sim.close()
    serve = serving(args) if (args.serve and rank == 0) else None

    if rank != 0:
        return
    cb = None if args.no_cpu else cpu_baseline(args, meta)
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp32_coloured": "f32",
                                                           "fp32_fixed64": "f32+i64", "fp64": "f64"}[args.precision],
        "data": "synthetic", "config": meta,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                     "frac": ach / hbm, "peak_source": which,
                     "traffic": measured_traffic(dom, args.config, dim, int(p.cfg["degree"]), args.precision,
                                                 args.ppa, n_p, tile_of(args)),
                     "k1_k2_k3_gbs": k123_gbs, "k1_k2_k3_frac": k123_gbs / hbm,
                     "k1_k2_k3_frac_nominal_7.7TB": k123_gbs / NOMINAL_HBM},
        "phase_ms_per_step": {"p2g": per_launch_ms["p2g"], "grid_g2p": per_launch_ms["grid_g2p"],
                              "g2pd": per_launch_ms["g2pd"], "time_advance": phase_ms[3] / prof_steps,
                              "reorder": phase_ms[4] / prof_steps, "profiled_steps": prof_steps},
        "algorithmic_bytes": alg,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": ck,
        # physical time the timed steps advanced (CFL steps), and the device
        # time per simulated second (the paper's wall-time figure, Sec. 4.3)
        "sim_time": {"simulated_s": t_sim1 - t_sim0,
                     "device_s_per_simulated_s": (ms / 1e3) / (t_sim1 - t_sim0) if t_sim1 > t_sim0 else None},
        "e2e": e2e,
        "cpu_baseline": cb,
    }
    if serve:
        line["serving"] = serve
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def end_to_end(M, p, args):
    """Same metric through the C ABI from host buffers: create, H2D of the
    initial state (page-locked before the timed region; binary32 arrays
    through mpm_add_particles_f32 for the FP32 modes, which store it in that
    precision, doubles for FP64), K steps, D2H of the density field (into a
    page-locked array) and of the FP64 conservation sums."""
    import dataclasses
    import torch

    f32 = args.precision.startswith("fp32")

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float32 if f32 else torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t

    host = {k: pinned(getattr(p, k)) for k in ("x", "v", "mass", "rho", "e")}
    q = dataclasses.replace(p, **{k: t.numpy() for k, t in host.items()})
    out = torch.empty(p.n_particles, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = M.Simulation.from_problem(q, f32=f32)
    sim.step(args.steps)
    rho = sim.read("RHO", out=out.numpy())
    cons = sim.conservation()
    t1 = time.perf_counter()
    sim.close()
    n = p.n_particles
    d = p.cfg["dim"]
    h2d = n * (2 * d + 3) * (4 if f32 else 8) + (p.mask.nbytes + p.normals.nbytes if p.mask is not None else 0)
    d2h = rho.nbytes + cons.nbytes
    return {"value": n * args.steps / (t1 - t0), "unit": "particle-steps/s",
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
            "seconds": t1 - t0}


if __name__ == "__main__":
    main()
