"""Continuous-batching request loop over many independent MPM simulations.

Requests (independent problems of different sizes) arrive over time.  A
request is admitted as soon as it has arrived and its device memory fits in
the remaining HBM budget; its state then stays resident on the GPU until it
finishes.  All admitted problems are members of one batch (mpm_batch_*): each
stage of a step is one launch over the flattened list of (problem, tile)
pairs, one step of the whole batch is a recorded CUDA graph, and the batch
advances in chunks of steps.  When a chunk completes, problems that have done
their steps are read back and retired at once, freeing memory for waiting
requests, which join before the next chunk.  Tile shapes come from the tile
tuner (tune.py) when one is given.

The baseline `run_sequential` solves the same requests one at a time in
arrival order with the same kernels and tile shapes.  Both report solves/s
and the p50/p99 latency from arrival to the result on the host.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import inputs as I
from . import mpm as M


def footprint_bytes(prob) -> int:
    """Device bytes a problem holds while resident: two particle buffers of
    2 n + 95 x tiles slots (every tile owns a region with room to grow; tiles
    hold at least 32 spans), the initial sort's scratch, grid accumulators,
    masks, per-span and per-tile tables."""
    cfg = prob.cfg
    d = int(cfg["dim"])
    p = int(cfg["degree"])
    real = 8 if cfg.get("precision") == "fp64" else 4
    acc = 4 if cfg.get("precision", "fp32") in ("fp32", "fp32_coloured") else 8
    n = prob.n_particles
    nodes = 1
    spans = 1
    for a in range(d):
        per = cfg["bc"][2 * a] in ("periodic", 1)
        nodes *= (cfg["n"][a] if per else cfg["n"][a] + 2 * p - 1) + 3
        spans *= cfg["n"][a] + 1 + 64
    tiles = spans // 32 + 1
    slots = 2 * n + 95 * tiles
    part = 2 * slots * ((2 * d + 4) * real + 12) + 4 * n * 4 + n * 8
    grid = (1 + 3 * d) * nodes * acc + nodes * (1 + d * real)
    return int(part + grid + 12 * spans + 32 * tiles + (1 << 20))


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    particles: int
    steps: int
    rho: np.ndarray | None
    ids: np.ndarray | None
    conservation: np.ndarray | None
    error: str = ""

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def _summary(results: list[Result], t0: float, t1: float) -> dict:
    ok = [r for r in results if not r.error]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    ps = sum(r.particles * r.steps for r in ok)
    return {"solves": len(ok), "failed": len(results) - len(ok), "seconds": t1 - t0,
            "solves_per_s": len(ok) / (t1 - t0), "particle_steps_per_s": ps / (t1 - t0),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "errors": sorted({r.error for r in results if r.error})}


def _failed(req, arrival, admitted, n, steps, err: str) -> Result:
    return Result(req["id"], arrival, admitted, time.perf_counter(), n, steps, None, None, None, err)


def _finish(sim, req, arrival, admitted, n, steps) -> Result:
    ids = sim.read("ID").astype(np.int64)
    rho = sim.read("RHO")
    cons = sim.conservation()
    return Result(req["id"], arrival, admitted, time.perf_counter(), n, steps, rho, ids, cons)


class Server:
    """Continuous batching over one mpm_batch: admission by HBM budget, state
    resident on the device, all members advanced together chunk by chunk."""

    def __init__(self, hbm_budget: float = 120e9, chunk: int = 25, max_active: int = 256, tuner=None):
        self.budget = float(hbm_budget)
        self.chunk = int(chunk)
        self.max_active = int(max_active)
        self.tuner = tuner

    def run(self, requests: list[dict], realtime: bool = True) -> tuple[list[Result], dict]:
        import torch
        reqs = sorted(requests, key=lambda r: r["arrival"])
        pending: list[dict] = []                       # arrived, problem not built yet
        waiting: list[tuple[dict, object, int]] = []   # built, not admitted yet
        active: list[dict] = []
        results: list[Result] = []
        used = 0.0
        nxt = 0
        batch = M.Batch()
        ev = None
        t0 = time.perf_counter()
        try:
            while nxt < len(reqs) or pending or waiting or active:
                now = time.perf_counter() - t0
                # arrivals (all at once when not in real time)
                while nxt < len(reqs) and (not realtime or reqs[nxt]["arrival"] <= now):
                    pending.append(reqs[nxt])
                    nxt += 1
                busy = ev is not None and not ev.query()
                # build the arrived problems on the host while the device runs
                # a chunk, or when there is nothing to admit or run
                if pending and len(waiting) < self.max_active and (busy or (not active and not waiting)):
                    waiting.append(self._build(pending.pop(0)))
                    continue
                if busy:
                    time.sleep(0.0002)
                    continue
                if ev is not None:
                    # a chunk has completed: account it, retire finished members
                    ev = None
                    try:
                        batch.sync()
                    except M.MPMError:
                        active = self._drop_failed(batch, active, results)
                        used = sum(a["bytes"] for a in active)
                    still = []
                    for a in active:
                        a["left"] -= a["running"]
                        a["running"] = 0
                        if a["left"] <= 0:
                            batch.remove(a["sim"])
                            results.append(_finish(a["sim"], a["req"], a["arrival"], a["admitted"], a["n"],
                                                   a["steps"]))
                            a["sim"].close()
                            used -= a["bytes"]
                        else:
                            still.append(a)
                    active = still
                # admission in arrival order while memory and slots allow
                while waiting and len(active) < self.max_active and used + waiting[0][2] <= self.budget:
                    r, prob, fb = waiting.pop(0)
                    sim = M.Simulation.from_problem(prob)
                    batch.add(sim, prob.steps)
                    arrival = t0 + (r["arrival"] if realtime else 0.0)
                    active.append({"req": r, "sim": sim, "left": prob.steps, "running": 0, "bytes": fb,
                                   "arrival": arrival, "admitted": time.perf_counter(), "n": prob.n_particles,
                                   "steps": prob.steps})
                    used += fb
                if active:
                    k = min(self.chunk, max(a["left"] for a in active))
                    batch.step_async(k)
                    for a in active:
                        a["running"] = k
                    ev = torch.cuda.Event()
                    ev.record(torch.cuda.ExternalStream(batch.stream))
                elif waiting and used == 0 and waiting[0][2] > self.budget:
                    raise RuntimeError("request larger than the HBM budget")
                else:
                    time.sleep(0.0002)
        finally:
            batch.close()
        t1 = time.perf_counter()
        return results, _summary(results, t0, t1)

    def _build(self, r):
        prob = I.request_problem(r)
        if self.tuner is not None:
            prob.cfg["tile"] = self.tuner.tile_for(prob)
        return r, prob, footprint_bytes(prob)

    @staticmethod
    def _drop_failed(batch, active, results):
        """A member raised an error (its state is then poisoned): take every
        member out, retire the failed ones with their error, put the others
        back with the steps they have left."""
        keep = []
        for a in active:
            batch.remove(a["sim"])
            try:
                a["sim"].sync()
            except M.MPMError as e:
                results.append(_failed(a["req"], a["arrival"], a["admitted"], a["n"], a["steps"], e.status))
                a["sim"].close()
                continue
            keep.append(a)
        for a in keep:
            # budget after the chunk that has just completed (the caller then
            # accounts that chunk); a finished member is retired before any
            # further step, so a budget of one is never used
            batch.add(a["sim"], max(a["left"] - a["running"], 1))
        return keep


def run_sequential(requests: list[dict], realtime: bool = True, tuner=None) -> tuple[list[Result], dict]:
    """One request at a time in arrival order with the same kernels; the next
    arrived request's problem is built on the host while the current one
    runs, as the batched server does."""
    reqs = sorted(requests, key=lambda r: r["arrival"])
    results = []
    t0 = time.perf_counter()

    def build(r):
        if realtime:
            wait = r["arrival"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        prob = I.request_problem(r)
        if tuner is not None:
            prob.cfg["tile"] = tuner.tile_for(prob)
        return prob

    nxt = build(reqs[0]) if reqs else None
    for i, r in enumerate(reqs):
        prob = nxt
        admitted = time.perf_counter()
        sim = M.Simulation.from_problem(prob)
        arrival = t0 + (r["arrival"] if realtime else 0.0)
        err = None
        try:
            sim.step_async(prob.steps)
        except M.MPMError as e:
            err = e
        arrived = i + 1 < len(reqs) and (not realtime or reqs[i + 1]["arrival"] <= time.perf_counter() - t0)
        nxt = build(reqs[i + 1]) if arrived else None
        if err is None:
            try:
                sim.sync()
            except M.MPMError as e:
                err = e
        if err is None:
            results.append(_finish(sim, r, arrival, admitted, prob.n_particles, prob.steps))
        else:
            results.append(_failed(r, arrival, admitted, prob.n_particles, prob.steps, err.status))
        sim.close()
        if nxt is None and i + 1 < len(reqs):
            nxt = build(reqs[i + 1])
    t1 = time.perf_counter()
    return results, _summary(results, t0, t1)
