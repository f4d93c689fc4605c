"""Tile-shape autotuner.

The step kernels give one CTA one tile of spans, so the tile shape sets the
particles per block, the shared-memory window (tile + halo nodes) and the
re-order's neighbourhood.  The best shape depends on the problem's
dimension, basis degree, precision and size.  `TileTuner.tile_for(prob)`
times each valid candidate on the problem itself (a few steps, CUDA events on
the simulation's stream, after warm-up steps) the first time a problem of
its class is seen, and returns the fastest shape from then on.  The class is
(dimension, degree, precision, periodic axes, log2 of the particle count);
decisions are kept in memory and, if a path is given, in a JSON file.
"""
from __future__ import annotations

import json
import math
import os

from . import mpm as M

CANDIDATES = {
    2: [(32, 8, 1), (32, 4, 1), (16, 8, 1), (16, 16, 1), (64, 4, 1), (32, 16, 1), (64, 8, 1)],
    3: [(16, 8, 4), (16, 4, 8), (8, 8, 8), (32, 4, 4), (16, 4, 4), (8, 16, 4), (32, 8, 2)],
}


class TileTuner:
    def __init__(self, steps: int = 4, warmup: int = 2, path: str | None = None, candidates=None):
        self.steps = int(steps)
        self.warmup = int(warmup)
        self.path = path
        self.candidates = candidates or CANDIDATES
        self.table: dict[str, list[int]] = {}
        self.timings: dict[str, dict[str, float]] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = {k: list(v) for k, v in json.load(f).items()}

    @staticmethod
    def problem_class(prob) -> str:
        cfg = prob.cfg
        per = "".join("p" if cfg["bc"][2 * a] in ("periodic", 1) else "n" for a in range(cfg["dim"]))
        size = int(round(math.log2(max(prob.n_particles, 1))))
        return f"d{cfg['dim']}-p{cfg.get('degree', 2)}-{cfg.get('precision', 'fp32')}-{per}-n2^{size}"

    def time_tile(self, prob, tile) -> float | None:
        """Milliseconds per step of `prob` with this tile, or None if invalid."""
        import torch
        cfg = dict(prob.cfg, tile=list(tile))
        try:
            sim = M.Simulation(cfg)
        except M.MPMError:
            return None
        try:
            sim.add_particles(prob.x, prob.v, prob.mass, prob.rho, prob.e)
            if prob.mask is not None:
                sim.set_obstacle_mask(prob.mask, prob.normals)
            sim.step(self.warmup)
            st = torch.cuda.ExternalStream(sim.stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sim.step_async(self.steps)
            e1.record(st)
            sim.sync()
            e1.synchronize()
            return e0.elapsed_time(e1) / self.steps
        except M.MPMError:
            return None
        finally:
            sim.close()

    def tile_for(self, prob) -> list[int]:
        key = self.problem_class(prob)
        if key in self.table:
            return list(self.table[key])
        best, best_ms, times = None, math.inf, {}
        for tile in self.candidates[int(prob.cfg["dim"])]:
            ms = self.time_tile(prob, tile)
            times["x".join(map(str, tile))] = ms
            if ms is not None and ms < best_ms:
                best, best_ms = list(tile), ms
        if best is None:
            best = [0, 0, 0]        # library default
        self.table[key] = best
        self.timings[key] = times
        if self.path:
            with open(self.path, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)
        return list(best)
