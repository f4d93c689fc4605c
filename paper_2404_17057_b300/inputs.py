"""Seeded synthetic inputs for the MPM hot path (shared by the CUDA path and the oracle).

This module only builds initial conditions -- particle positions, masses,
densities, internal energies and the obstacle node mask/normals -- with the
shapes and distributions of the paper's test cases (Sec. 4.1):

* ``shock_tube``  -- Sod tube, quasi-1D strip, regular 2x2 lattice per cell;
* ``cylinder``    -- Mach-M flow past a cylinder, stratified random positions
                     (one uniform point per sub-cell, Sec. 4.1 prefers random
                     placement), inflow/outflow/slip walls, obstacle as a node
                     mask with analytic normals n = grad sd;
* ``blast``       -- 3D point blast: ambient gas at rest, energy deposited in
                     the particles near the centre, reflective walls;
* ``uniform_flow``/``linear_velocity`` -- states with closed-form evolution;
* ``serving_stream`` -- a seeded list of independent problems.

No step of the method is evaluated here.  Node arrays use the library's node
storage layout: along a non-periodic axis a degree-p grid stores n + 2p - 1
nodes, node i at origin + (i - (p - 1)) h; a periodic axis stores n nodes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class Problem:
    name: str
    cfg: dict
    x: np.ndarray            # (d, N) float64
    v: np.ndarray            # (d, N)
    mass: np.ndarray         # (N,)
    rho: np.ndarray
    e: np.ndarray            # specific internal energy
    mask: np.ndarray | None = None      # (nodes,) uint8
    normals: np.ndarray | None = None   # (d, nodes) float64
    steps: int = 0
    t_end: float = 0.0
    meta: dict = field(default_factory=dict)
    profile: list | None = None         # closed loops of obstacle boundary points, (2, k) each

    @property
    def n_particles(self) -> int:
        return int(self.mass.shape[0])


def base_config(dim, n, h, bc, degree=2, **kw) -> dict:
    cfg = {"dim": dim, "n": list(n), "h": float(h), "origin": [0.0, 0.0, 0.0], "gamma": 1.4,
           "c0": 1.0, "c1": 1.0, "degree": degree, "bc": list(bc), "inflow_rho": 1.0,
           "inflow_p": 1.0, "inflow_v": [0.0, 0.0, 0.0], "cfl": 0.4, "sort_interval": 1,
           "seed": 0, "tile": [0, 0, 0], "precision": "fp32", "fixed_unit": [0.0, 0.0, 0.0]}
    cfg.update(kw)
    return cfg


def node_shape(cfg: dict):
    """Number of stored nodes per axis and the storage offset of physical node 0."""
    p = int(cfg["degree"])
    shape, off = [], []
    for a in range(int(cfg["dim"])):
        per = cfg["bc"][2 * a] in ("periodic", 1)
        n = int(cfg["n"][a])
        shape.append(n if per else n + 2 * p - 1)
        off.append(0 if per else p - 1)
    return shape, off


def node_coords(cfg: dict):
    """Physical coordinates of every stored node, (d, nodes), x fastest."""
    shape, off = node_shape(cfg)
    h = cfg["h"]
    axes = [cfg["origin"][a] + (np.arange(shape[a]) - off[a]) * h for a in range(len(shape))]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    return np.stack([g.reshape(-1) for g in grids])


def _lattice(n, h, ppa, dim, lo=None):
    """Regular lattice, ppa points per axis per cell at offsets (a + 1/2)/ppa."""
    lo = lo or [0.0] * dim
    axes = [lo[a] + (np.arange(n[a] * ppa) + 0.5) * (h / ppa) for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    return np.stack([g.reshape(-1) for g in grids])


def _stratified(n, h, ppa, dim, rng, lo=None):
    """One uniform random point in each of the ppa^d sub-cells of every cell."""
    lo = lo or [0.0] * dim
    base = _lattice(n, h, ppa, dim, lo) - 0.5 * (h / ppa)
    return base + rng.random(base.shape) * (h / ppa)


def shock_tube(ncell=200, ny=4, degree=2, ppa=2, t_end=0.2, precision="fp64", x0=0.5,
               left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), cfl=0.4, **kw) -> Problem:
    """Sod tube on [0,1] x [0, ny h] (Sec. 4.1): walls in x, periodic in y."""
    h = 1.0 / ncell
    cfg = base_config(2, [ncell, ny], h, ["wall", "wall", "periodic", "periodic"], degree=degree,
                      cfl=cfl, precision=precision, **kw)
    x = _lattice([ncell, ny], h, ppa, 2)
    N = x.shape[1]
    isl = x[0] < x0
    rho = np.where(isl, left[0], right[0])
    p = np.where(isl, left[2], right[2])
    v = np.zeros((2, N))
    v[0] = np.where(isl, left[1], right[1])
    mass = rho * h * h / (ppa * ppa)
    e = p / ((cfg["gamma"] - 1.0) * rho)
    return Problem("shock_tube", cfg, x, v, mass, rho, e, t_end=t_end,
                   meta={"left": left, "right": right, "x0": x0})


def cylinder_mask(cfg: dict, center, radius):
    """Node mask and normals for a cylinder (sd(x) = |x - c| - r).

    A cell is an obstacle cell when one of its corners has sd <= 0; the corner
    nodes of obstacle cells are masked; n_i = grad sd(x_i) = (x_i - c)/|x_i - c|
    (zero at the centre)."""
    shape, off = node_shape(cfg)
    h = cfg["h"]
    nx, ny = cfg["n"][0], cfg["n"][1]
    cx, cy = center
    cells_x = np.arange(nx)
    cells_y = np.arange(ny)
    X0 = (cells_x[None, :]) * h + cfg["origin"][0]
    Y0 = (cells_y[:, None]) * h + cfg["origin"][1]
    inside = np.zeros((ny, nx), dtype=bool)
    for dx in (0, 1):
        for dy in (0, 1):
            inside |= np.hypot(X0 + dx * h - cx, Y0 + dy * h - cy) <= radius
    mask = np.zeros((shape[1], shape[0]), dtype=np.uint8)
    jj, ii = np.nonzero(inside)
    for dx in (0, 1):
        for dy in (0, 1):
            mask[jj + dy + off[1], ii + dx + off[0]] = 1
    xy = node_coords(cfg)
    dx = xy[0] - cx
    dy = xy[1] - cy
    r = np.hypot(dx, dy)
    with np.errstate(invalid="ignore", divide="ignore"):
        nrm = np.where(r > 0, np.stack([dx / r, dy / r]), 0.0)
    mask = mask.reshape(-1)
    nrm = np.where(mask[None, :] != 0, nrm, 0.0)
    return mask, np.ascontiguousarray(nrm)


def cylinder(nx=1024, ny=512, lx=2.0, center=(0.4, 0.5), radius=0.05, mach=3.0, rho0=1.4, p0=1.0,
             ppa=2, seed=1, steps=2000, degree=2, precision="fp32", cfl=0.4, mirrored=False,
             **kw) -> Problem:
    """Supersonic flow past a cylinder (Sec. 4.1): free stream everywhere at t=0,
    inflow on -x, outflow on +x with recycling, slip walls on +-y."""
    h = lx / nx
    cfg = base_config(2, [nx, ny], h, ["inflow", "outflow", "wall", "wall"], degree=degree, cfl=cfl,
                      inflow_rho=rho0, inflow_p=p0, inflow_v=[mach, 0.0, 0.0], seed=seed,
                      precision=precision, **kw)
    rng = np.random.default_rng(seed)
    if mirrored:
        assert ny % 2 == 0
        half = _stratified([nx, ny // 2], h, ppa, 2, rng)
        ly = ny * h
        x = np.concatenate([half, np.stack([half[0], ly - half[1]])], axis=1)
    else:
        x = _stratified([nx, ny], h, ppa, 2, rng)
    keep = np.hypot(x[0] - center[0], x[1] - center[1]) >= radius
    x = np.ascontiguousarray(x[:, keep])
    N = x.shape[1]
    rho = np.full(N, rho0)
    v = np.zeros((2, N))
    v[0] = mach
    mass = rho * h * h / (ppa * ppa)
    e = np.full(N, p0 / ((cfg["gamma"] - 1.0) * rho0))
    mask, nrm = cylinder_mask(cfg, center, radius)
    return Problem("cylinder", cfg, x, v, mass, rho, e, mask=mask, normals=nrm, steps=steps,
                   meta={"center": center, "radius": radius, "mach": mach})


def naca4_symmetric(thickness=0.12, chord=0.1, npts=200, alpha_deg=0.0, leading_edge=(0.0, 0.0)):
    """Closed boundary loop (2, 2 npts - 1) of a symmetric NACA 4-digit
    aerofoil: half-thickness y_t = 5 t c (0.2969 sqrt(s) - 0.1260 s - 0.3516 s^2
    + 0.2843 s^3 - 0.1015 s^4) at s = x/c (the published 4-digit series
    formula), cosine-spaced s, upper surface from the trailing edge to the
    nose, lower surface back (counter-clockwise); the loop closes across the
    blunt trailing edge.  Pitched nose-up by alpha about the leading edge.  Stands in for the OAT15a point file of the
    aerofoil case, which is not available."""
    s = 0.5 * (1.0 - np.cos(np.linspace(0.0, np.pi, npts)))
    yt = 5.0 * thickness * chord * (0.2969 * np.sqrt(s) - 0.1260 * s - 0.3516 * s ** 2 + 0.2843 * s ** 3
                                    - 0.1015 * s ** 4)
    xs = s * chord
    upper = np.stack([xs[::-1], yt[::-1]])
    lower = np.stack([xs[1:], -yt[1:]])
    loop = np.concatenate([upper, lower], axis=1)
    a = -np.deg2rad(alpha_deg)
    rot = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    return rot @ loop + np.asarray(leading_edge, dtype=np.float64)[:, None]


def inside_loops(x, loops):
    """Even-odd point-in-polygon test of points (2, N) against closed loops
    (used to leave no particle inside an obstacle)."""
    inside = np.zeros(x.shape[1], dtype=bool)
    for loop in loops:
        a = np.asarray(loop, dtype=np.float64)
        b = np.roll(a, -1, axis=1)
        for k in range(a.shape[1]):
            ax, ay, bx, by = a[0, k], a[1, k], b[0, k], b[1, k]
            cross = (ay > x[1]) != (by > x[1])
            with np.errstate(divide="ignore", invalid="ignore"):
                xc = ax + (x[1] - ay) * (bx - ax) / (by - ay)
            inside ^= cross & (x[0] < xc)
    return inside


def aerofoil(nx=600, ny=405, lx=0.4, mach=0.73, alpha_deg=25.0, chord=0.1, leading_edge=(0.1, 0.15),
             rho0=1.4, p0=1.0, ppa=3, npts=200, seed=2, steps=1000, degree=2, precision="fp32", cfl=0.4,
             **kw) -> Problem:
    """Transonic flow past an aerofoil (Sec. 4.1): [0, 0.4] x [0, 0.27], inflow
    at -x with v = (Mach, 0) (c = 1 for rho = 1.4, p = 1), outflow on the other
    faces, free stream everywhere at t = 0, 3 x 3 stratified ppc (9 ppc, about
    2.2M particles at 600 x 405 = 243k cells); the obstacle is a NACA 0012
    profile (stand-in for the OAT15a point file) at angle of attack alpha,
    handed to the library as a point loop."""
    h = lx / nx
    cfg = base_config(2, [nx, ny], h, ["inflow", "outflow", "outflow", "outflow"], degree=degree, cfl=cfl,
                      inflow_rho=rho0, inflow_p=p0, inflow_v=[mach, 0.0, 0.0], seed=seed,
                      precision=precision, **kw)
    loop = naca4_symmetric(0.12, chord, npts, alpha_deg, leading_edge)
    rng = np.random.default_rng(seed)
    x = _stratified([nx, ny], h, ppa, 2, rng)
    x = np.ascontiguousarray(x[:, ~inside_loops(x, [loop])])
    N = x.shape[1]
    rho = np.full(N, rho0)
    v = np.zeros((2, N))
    v[0] = mach
    mass = rho * h * h / (ppa * ppa)
    e = np.full(N, p0 / ((cfg["gamma"] - 1.0) * rho0))
    return Problem("aerofoil", cfg, x, v, mass, rho, e, steps=steps, profile=[loop],
                   meta={"mach": mach, "alpha_deg": alpha_deg, "chord": chord})


def blast(n=256, ppa=2, energy=1.0, rho0=1.0, p0=1e-5, steps=200, degree=2, precision="fp32",
          cfl=0.3, radius_cells=2.0, **kw) -> Problem:
    """3D point blast in the unit cube with reflective (slip) walls: ambient gas
    at rest; the particles with |X - c| < radius_cells*h share the energy
    `energy` as equal specific internal energy increments."""
    h = 1.0 / n
    cfg = base_config(3, [n, n, n], h, ["wall"] * 6, degree=degree, cfl=cfl, precision=precision, **kw)
    x = _lattice([n, n, n], h, ppa, 3)
    N = x.shape[1]
    rho = np.full(N, rho0)
    mass = np.full(N, rho0 * h ** 3 / ppa ** 3)
    e = np.full(N, p0 / ((cfg["gamma"] - 1.0) * rho0))
    r = np.sqrt(((x - 0.5) ** 2).sum(axis=0))
    hot = r < radius_cells * h
    e[hot] += energy / mass[hot].sum()
    v = np.zeros((3, N))
    return Problem("blast", cfg, x, v, mass, rho, e, steps=steps,
                   meta={"energy": energy, "hot": int(hot.sum())})


def uniform_flow(dim=2, n=(16, 16, 16), ppa=2, vel=(0.3, -0.2, 0.1), rho0=1.0, p0=1.0, degree=2,
                 precision="fp64", cfl=0.4, shift=0.0, **kw) -> Problem:
    """Uniform state on a periodic lattice: the exact solution keeps rho, v, e
    and translates X by v t."""
    n = list(n)[:dim]
    h = 1.0 / n[0]
    cfg = base_config(dim, n, h, ["periodic"] * (2 * dim), degree=degree, cfl=cfl, precision=precision, **kw)
    x = _lattice(n, h, ppa, dim) + shift * h
    L = np.array([n[a] * h for a in range(dim)])[:, None]
    x = np.mod(x, L)
    N = x.shape[1]
    v = np.tile(np.array(vel[:dim])[:, None], (1, N))
    rho = np.full(N, rho0)
    mass = np.full(N, rho0 * h ** dim / ppa ** dim)
    e = np.full(N, p0 / ((cfg["gamma"] - 1.0) * rho0))
    return Problem("uniform_flow", cfg, x, v, mass, rho, e)


def linear_velocity(dim=2, n=16, ppa=2, a=0.05, degree=2, precision="fp64", e0=0.0, rho0=1.0, **kw) -> Problem:
    """Gas of uniform density rho0 and internal energy e0 with V = a X on a
    lattice, free (outflow) faces: interior particles see div V = d a."""
    h = 1.0 / n
    cfg = base_config(dim, [n] * dim, h, ["outflow"] * (2 * dim), degree=degree, precision=precision, **kw)
    x = _lattice([n] * dim, h, ppa, dim)
    N = x.shape[1]
    v = a * x
    rho = np.full(N, float(rho0))
    mass = np.full(N, rho0 * h ** dim / ppa ** dim)
    e = np.full(N, float(e0))
    return Problem("linear_velocity", cfg, x, v, mass, rho, e, meta={"a": a})


def serving_stream(count=512, seed=5, steps=500, rate=50.0, side_lo=64, side_hi=1024,
                   precision="fp32_fixed64", max_side=None) -> list[dict]:
    """Independent 2D problems: kind in {shock tube, cylinder} with probability
    1/2; side n log-uniform on [side_lo, side_hi] rounded to a multiple of 16;
    cylinder radius U[0.02, 0.1], Mach U[1.5, 4]; Poisson arrivals."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        kind = "shock_tube" if rng.random() < 0.5 else "cylinder"
        side = math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))
        side = max(16, int(round(side / 16.0)) * 16)
        if max_side:
            side = min(side, max_side)
        req = {"id": i, "arrival": t, "kind": kind, "side": side, "steps": steps, "precision": precision}
        if kind == "cylinder":
            req["radius"] = float(rng.uniform(0.02, 0.1))
            req["mach"] = float(rng.uniform(1.5, 4.0))
            req["seed"] = int(rng.integers(1, 2 ** 31))
        out.append(req)
    return out


def request_problem(req: dict) -> Problem:
    """The Problem of one serving request."""
    n = int(req["side"])
    if req["kind"] == "shock_tube":
        p = shock_tube(ncell=n, ny=4, precision=req["precision"], t_end=0.0)
        p.cfg["n"] = [n, 4]
        p.cfg["h"] = 1.0 / n
    else:
        p = cylinder(nx=n, ny=n // 2, radius=req["radius"], mach=req["mach"], seed=req["seed"],
                     precision=req["precision"], steps=req["steps"])
    p.steps = int(req["steps"])
    if "cfl" in req:
        p.cfg["cfl"] = float(req["cfl"])
    if req["precision"] == "fp32_fixed64":
        p.cfg["fixed_unit"] = normalised_fixed_units(p)
    return p


MASS_UNIT_PER_PARTICLE = 8.0


def normalised_fixed_units(p) -> list[float]:
    """Fixed-point units scaled to the problem (the normalised reading of the
    'scale 2^-32 per unit' option): mass unit = 8 x the mean particle mass,
    momentum unit = mass unit x (|v| + c) of the faster of the two states,
    force unit = momentum unit / the first CFL step.  A contribution of one
    particle then spans about 2^29 quanta, whatever the resolution: still 32
    times finer than binary32, and below 2^31, where the P2G quantises with
    32-bit conversions."""
    cfg = p.cfg
    g = float(cfg.get("gamma", 1.4))
    um = MASS_UNIT_PER_PARTICLE * float(np.mean(p.mass))
    c = np.sqrt(np.maximum(g * (g - 1.0) * p.e, 0.0))
    s = float(np.max(np.sqrt((p.v ** 2).sum(axis=0)) + c))
    umom = um * s
    dt0 = float(cfg.get("cfl", 0.4)) * float(cfg["h"]) / s
    return [um, umom, umom / dt0]
