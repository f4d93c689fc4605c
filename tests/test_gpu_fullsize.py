"""Full-size parity in the benchmark's launch configuration, on sampled outputs.

The 256^3 blast (134,217,728 particles, FP32) and the 1024x512 Mach-3
cylinder (FP32) run one step on the GPU with the kernels and launch shapes the
benchmark times.  One step of a particle depends only on particles within a
few cells of it (P2G support 1.5 h, grid velocity of those nodes, second P2G,
G2PD), so the oracle recomputes sampled particles one by one on a box of
+-8 cells of the same initial state around each sample (grid-aligned, true
domain faces keep their boundary condition, cut faces impose none).  Both
sides use the same fixed dt.  Tolerance: the FP32 bound of the fields
(relative 2e-5 of the local scale) -- one step, no accumulated drift.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2404_17057_b300 import inputs as I
from paper_2404_17057_b300 import mpm as M

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HALF = 8   # box half-width in cells


def local_box(p, k, dt):
    """Oracle simulation of the particles within HALF cells of particle k."""
    cfg = dict(p.cfg)
    d = cfg["dim"]
    h = cfg["h"]
    xk = p.x[:, k]
    lo_c = [max(0, int(np.floor(xk[a] / h)) - HALF) for a in range(d)]
    hi_c = [min(cfg["n"][a], int(np.floor(xk[a] / h)) + HALF + 1) for a in range(d)]
    sel = np.ones(p.n_particles, dtype=bool)
    for a in range(d):
        sel &= (p.x[a] >= lo_c[a] * h) & (p.x[a] <= hi_c[a] * h)
    idx = np.nonzero(sel)[0]
    bc = []
    for a in range(d):
        bc.append(cfg["bc"][2 * a] if lo_c[a] == 0 else "outflow")
        bc.append(cfg["bc"][2 * a + 1] if hi_c[a] == cfg["n"][a] else "outflow")
    sub = dict(cfg, n=[hi_c[a] - lo_c[a] for a in range(d)], origin=[lo_c[a] * h for a in range(d)] + [0.0] * (3 - d),
               bc=bc, precision="fp64")
    if "inflow" not in bc:
        sub["inflow_rho"] = cfg["inflow_rho"]
    s = O.OracleSim(sub)
    s.add_particles(p.x[:, idx], p.v[:, idx], p.mass[idx], p.rho[idx], p.e[idx])
    if p.mask is not None:
        s.set_obstacle_mask(*sub_mask(p, cfg, sub, lo_c))
    s.step(1, dt=dt)
    ids = s.read("ID").astype(np.int64)
    j = int(np.nonzero(idx[ids] == k)[0][0])
    out = {}
    for f in ("X", "V", "RHO", "E", "Q"):
        a = s.read(f)
        out[f] = (a[..., j], float(np.abs(a).max()))   # value and its scale over the box
    return out


def sub_mask(p, cfg, sub, lo_c):
    shape, off = I.node_shape(cfg)
    sshape, soff = I.node_shape(sub)
    d = cfg["dim"]
    m = p.mask.reshape(shape[::-1])
    nrm = p.normals.reshape((d,) + tuple(shape[::-1]))
    # physical node index i of the box is node lo_c + i of the domain
    sl = tuple(slice(lo_c[a] - soff[a] + off[a], lo_c[a] - soff[a] + off[a] + sshape[a]) for a in range(d))[::-1]
    return m[sl].reshape(-1).copy(), nrm[(slice(None),) + sl].reshape(d, -1).copy()


def f32(p):
    for k in ("x", "v", "mass", "rho", "e"):
        setattr(p, k, getattr(p, k).astype(np.float32).astype(np.float64))
    return p


def check(p, dt, samples):
    p = f32(p)
    g = M.Simulation.from_problem(p)
    g.step(1, dt=dt)
    ids = g.read("ID").astype(np.int64)
    inv = np.empty_like(ids)
    inv[ids] = np.arange(ids.shape[0])
    got = {f: g.read(f) for f in ("X", "V", "RHO", "E", "Q")}
    g.close()
    for k in samples:
        ref = local_box(p, k, dt)
        j = inv[k]
        for f in ("X", "V", "RHO", "E", "Q"):
            a = got[f][..., j]
            b, scale = ref[f]
            # binary32: positions to a few ulps of the coordinate, other fields
            # to 2e-5 of their magnitude over the box
            # Q is proportional to div V, a cancelling sum of ~|v|/h terms, so its
            # binary32 error is relative to that scale rather than to Q itself
            floor = {"V": 1e-9, "RHO": 1e-9, "E": 1e-12, "Q": 1e-12}
            rel = 1e-4 if f == "Q" else 2e-5
            tol = 4e-7 * max(1.0, np.abs(b).max()) if f == "X" else rel * scale + floor[f]
            assert np.abs(a - b).max() <= tol, (k, f, a, b, tol)


def test_blast_256_full_size_sampled():
    p = I.blast(n=256)
    n = 256
    h = 1.0 / n
    c = 0.5
    # near the blast, inside the shell, at rest far away, at a wall and a corner
    pts = [(c + 0.3 * h, c, c), (c + 2.5 * h, c - 1.7 * h, c + 0.9 * h), (0.3, 0.7, 0.45),
           (0.25 * h, 0.5, 0.5), (0.999, 0.001, 0.998)]
    samples = [int(np.argmin(((p.x - np.array(q)[:, None]) ** 2).sum(axis=0))) for q in pts]
    # the energised particles have a sound speed near 500: dt below their CFL limit
    check(p, 1e-6, samples)


def test_cylinder_1024_full_size_sampled():
    p = I.cylinder(nx=1024, ny=512)
    h = p.cfg["h"]
    pts = [(0.4 - 0.05 - 1.5 * h, 0.5), (0.4, 0.5 + 0.05 + h), (1.0, 0.3), (0.5 * h, 0.2), (2.0 - 0.3 * h, 0.6),
           (1.3, 0.5 * h)]
    samples = [int(np.argmin(((p.x - np.array(q)[:, None]) ** 2).sum(axis=0))) for q in pts]
    check(p, 1e-4, samples)


def test_blast_front_follows_sedov_taylor_on_the_gpu():
    """The C3 physics of the FP32 GPU path on its own: a 64^3 blast's shock
    front is within 5% of the Sedov-Taylor radius xi0 (E t^2/rho)^(1/5) at
    t = 0.02..0.04 and grows as t^(2/5) (same measure as the oracle pin)."""
    from test_oracle_pins import _blast_front, _gold
    g = _gold("sedov_taylor.txt")
    xi0, ex = g["xi0_gamma_1_4"][0], g["exponent"][0]
    n = 64
    p = I.blast(n=n, radius_cells=1.5)
    s = M.Simulation.from_problem(p)
    fronts = {}
    for t in (0.02, 0.03, 0.04):
        s.step(100000, t_end=t)
        rf, peak = _blast_front(s, n)
        fronts[t] = rf
        assert abs(rf / (xi0 * t ** ex) - 1.0) < 0.05, (t, rf)
        assert 1.5 < peak < 6.0
    s.close()
    assert abs(fronts[0.04] / fronts[0.02] / 2.0 ** ex - 1.0) < 0.04


def _standoff(s, p):
    """Bow-shock standoff / R on the stagnation line: particles within 2h of
    the cylinder's axis line upstream of it, binned by h; the shock is where
    the density first passes half-way from the free stream to its peak
    (linear between bin centres)."""
    c, R, h = p.meta["center"], p.meta["radius"], p.cfg["h"]
    x, rho = s.read("X"), s.read("RHO")
    sel = (np.abs(x[1] - c[1]) < 2 * h) & (x[0] < c[0] - R)
    edges = np.arange(0.0, c[0] - R + 0.5 * h, h)
    idx = np.digitize(x[0][sel], edges) - 1
    prof = np.array([rho[sel][idx == i].mean() for i in range(len(edges) - 1)])
    mid = 0.5 * (edges[:-1] + edges[1:])
    rinf = p.rho[0]
    half = rinf + 0.5 * (prof.max() - rinf)
    j = int(np.argmax(prof > half))
    xs = mid[j - 1] + (half - prof[j - 1]) / (prof[j] - prof[j - 1]) * h
    return (c[0] - R - xs) / R


def test_cylinder_bow_shock_standoff_on_the_gpu():
    """The C2 physics of the FP32 GPU path on its own: the bow shock of the
    1024x512 Mach-3 cylinder (r = 0.05, 25.6 cells) stands off by Billig's
    Delta/R = 0.386 exp(4.67/M^2) = 0.648 within 20%, averaged over
    t = 0.35..0.55 once the shock has settled.  The half-rise front of a
    shock smeared over 2-3 cells (about 0.1 R) sits upstream of the
    discontinuity, so the measure reads high."""
    from test_oracle_pins import _gold
    g = _gold("bow_shock_standoff.txt")
    mach = 3.0
    ref = g["a_cylinder"][0] * np.exp(g["b_cylinder"][0] / mach ** 2)
    p = I.cylinder(nx=1024, ny=512, mach=mach)
    s = M.Simulation.from_problem(p)
    vals = []
    for t in (0.35, 0.40, 0.45, 0.50, 0.55):
        s.step(100000, t_end=t)
        vals.append(_standoff(s, p))
    s.close()
    assert abs(np.mean(vals) / ref - 1.0) < 0.2, vals
    assert np.std(vals) < 0.1, vals        # settled


def test_blast_256_twenty_steps_keep_mass_and_symmetry():
    """The 256^3 blast in the benchmark's launch configuration (8x8x8 tiles,
    FP32) for 20 CFL steps, checked by properties that hold at any size.
    Particle masses never change, and 2^27 equal binary32 masses sum exactly
    in binary64 in any order, so the FP64 mass sum stays N M bit for bit.
    The deposit and the walls are symmetric about the centre, so the total
    momentum stays zero up to the rounding of the float-atomic sums: below
    1e-5 of sum M |V|."""
    p = f32(I.blast(n=256, tile=[8, 8, 8]))
    g = M.Simulation.from_problem(p)
    m0 = g.conservation()[0]
    assert m0 == p.mass.shape[0] * p.mass[0]
    g.step(20)
    c = g.conservation()
    assert c[0] == m0
    mass, v = g.read("M"), g.read("V")
    scale = float((mass * np.sqrt((v ** 2).sum(axis=0))).sum())
    drift = np.abs(c[2:5]).max() / scale
    print("momentum / sum M|V| after 20 steps:", drift)
    assert scale > 0 and drift <= 1e-5, (c, scale)
    g.close()
