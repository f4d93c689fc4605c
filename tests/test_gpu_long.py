"""Drift over the C2 run length: the Mach-3 cylinder of Sec. 4.1 for 2000 steps.

C2 runs 2000 steps; the other whole-step tests against the oracle stop at 100.
Here a 128 x 64 cylinder of radius 0.15 (9.6 cells; 31,609 particles, inflow
recycling, obstacle mask) runs to t = 1.35, about 2000 steps, in the FP64
oracle and on the GPU in FP64 and in FP32 with float atomics, each stopping
at the same five times t = 1.15 .. 1.35 (equal times, not equal step counts:
the CFL step follows the largest particle speed).

By then the wake sheds vortices and particle trajectories are chaotic: FP64
on the GPU, which differs from the oracle only in the order of its sums,
leaves about 14% of the particles more than a cell from their oracle
positions, FP32 about 65%, and two GPU runs of the same problem differ from
each other as much (float atomics add in a different order each run).  So
the comparison is of what the flow keeps: the bow-shock standoff on the
stagnation line (the steady flow ahead of the body), averaged over the five
times, and the means of rho, P, e and |V|^2 over all particles at the last.
The FP32 path with float atomics adds in a different order each run, and in
this unsteady flow its averaged standoff spreads from run to run: measured on
a B300, 0.15-0.5% from the oracle's in most runs and 2.3% in one.  The two
FP32 modes that are bit-reproducible run to run (P2G in colour passes, and
int64 fixed point) give the same result every time, and FP64 differs from
the oracle only in the order of its sums (0.3-0.5%).  The means stayed
within 0.3% (FP64) and 1.4% (FP32).  Bounds: 2% for the averaged standoff
(5% for float-atomic FP32), 2.5% for the means.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2404_17057_b300 import inputs as I
from paper_2404_17057_b300 import mpm as M

pytestmark = pytest.mark.gpu

STEPS = 2000
RADIUS = 0.15


def f32(p):
    for k in ("x", "v", "mass", "rho", "e"):
        setattr(p, k, getattr(p, k).astype(np.float32).astype(np.float64))
    return p


def problem(precision):
    return f32(I.cylinder(nx=128, ny=64, seed=1, radius=RADIUS, precision=precision))


def standoff(x, rho, p):
    """Bow-shock standoff / R on the stagnation line: particles within 3h of
    the axis upstream of the body, binned by h; the shock is where the
    density first passes half-way from the free stream to its peak."""
    c, R, h = p.meta["center"], p.meta["radius"], p.cfg["h"]
    sel = (np.abs(x[1] - c[1]) < 3 * h) & (x[0] < c[0] - R)
    edges = np.arange(0.0, c[0] - R + 0.5 * h, h)
    idx = np.digitize(x[0][sel], edges) - 1
    prof = np.array([rho[sel][idx == i].mean() for i in range(len(edges) - 1)])
    mid = 0.5 * (edges[:-1] + edges[1:])
    half = p.rho[0] + 0.5 * (prof.max() - p.rho[0])
    j = int(np.argmax(prof > half))
    xs = mid[j - 1] + (half - prof[j - 1]) / (prof[j] - prof[j - 1]) * h
    return (c[0] - R - xs) / R


TIMES = (1.15, 1.20, 1.25, 1.30, 1.35)


def run(sim, p):
    """Standoffs at TIMES and the means at the last."""
    so = []
    for t in TIMES:
        sim.step(100000, t_end=t)
        so.append(standoff(sim.read("X"), sim.read("RHO"), p))
    out = summary(sim, p)
    out["standoff"] = float(np.mean(so))
    return out


def summary(sim, p):
    rho, v = sim.read("RHO"), sim.read("V")
    return {"RHO": rho.mean(), "P": sim.read("P").mean(), "E": sim.read("E").mean(),
            "V2": (v ** 2).sum(axis=0).mean()}


@pytest.fixture(scope="module")
def oracle_run():
    p = problem("fp64")
    o = O.OracleSim(p.cfg)
    o.add_particles(p.x, p.v, p.mass, p.rho, p.e)
    o.set_obstacle_mask(p.mask, p.normals)
    out = run(o, p)
    out["steps"] = int(o.read("CLOCK")[2])
    return out


# bound on the averaged standoff: the float-atomic FP32 path is the one whose
# result changes from run to run
STANDOFF_BOUND = {"fp64": 0.02, "fp32_coloured": 0.02, "fp32_fixed64": 0.02, "fp32": 0.05}


@pytest.mark.parametrize("precision", ["fp64", "fp32_coloured", "fp32_fixed64", "fp32"])
def test_cylinder_2000_steps_keeps_the_oracle_flow(oracle_run, precision):
    ref = oracle_run
    assert 1900 <= ref["steps"] <= 2100        # the C2 run length
    p = problem(precision)
    g = M.Simulation.from_problem(p)
    got = run(g, p)
    clock = g.read("CLOCK")
    assert abs(clock[0] - TIMES[-1]) <= 1e-12
    rel = {k: abs(got[k] / ref[k] - 1.0) for k in ("standoff", "RHO", "P", "E", "V2")}
    print(precision, int(clock[2]), "steps (oracle", ref["steps"], ")", got, rel)
    assert rel["standoff"] <= STANDOFF_BOUND[precision], (got, ref)
    for k in ("RHO", "P", "E", "V2"):
        assert rel[k] <= 0.025, (k, got, ref)
    g.close()
