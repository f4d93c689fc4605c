"""Obstacles from point profiles on the GPU (mpm_set_obstacle_profile)
against the oracle's evaluation of Eq. sdf and the obstacle-cell rule:
mask, normals and signed distance bit for bit, then a flow past the
profile against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2404_17057_b300 import inputs as I
from paper_2404_17057_b300 import mpm as M

pytestmark = pytest.mark.gpu


def _square(c, hw, ang_deg):
    a = np.deg2rad(ang_deg)
    rot = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    return rot @ np.array([[-hw, hw, hw, -hw], [-hw, -hw, hw, hw]]) + np.array(c)[:, None]


def _circle(c, r, k):
    th = 2 * np.pi * np.arange(k) / k
    return np.stack([c[0] + r * np.cos(th), c[1] + r * np.sin(th)])


CASES = [
    ("aerofoil", I.base_config(2, [120, 81], 0.4 / 120, ["inflow", "outflow", "outflow", "outflow"]),
     [I.naca4_symmetric(0.12, 0.1, 200, 25.0, (0.1, 0.15))]),
    ("square", I.base_config(2, [64, 48], 1 / 64, ["wall"] * 4, degree=1), [_square((0.47, 0.36), 0.17, 30.0)]),
    ("circle", I.base_config(2, [96, 64], 1 / 64, ["wall"] * 4), [_circle((0.71, 0.5), 0.2031, 4096)]),
    ("hole", I.base_config(2, [40, 40], 1 / 40, ["wall"] * 4),
     [_square((0.5, 0.5), 0.3, 0.0), _square((0.5, 0.5), 0.1, 0.0)]),
    ("periodic", I.base_config(2, [64, 32], 1 / 32, ["wall", "wall", "periodic", "periodic"]),
     [_circle((1.0, 0.5), 0.3, 300)]),
]


@pytest.mark.parametrize("name,cfg,loops", CASES, ids=[c[0] for c in CASES])
def test_profile_obstacle_is_the_oracle_bit_for_bit(name, cfg, loops):
    sim = M.Simulation(dict(cfg, precision="fp64"))
    mask, nrm, sd = sim.set_obstacle_profile(loops)
    om, on, osd = O.obstacle_profile(cfg, loops)
    assert np.array_equal(sd, osd)
    assert np.array_equal(mask, om)
    assert np.array_equal(nrm, on)
    assert mask.sum() > 20
    sim.close()


def test_profile_obstacle_errors():
    cfg = I.base_config(2, [64, 32], 1 / 64, ["inflow", "outflow", "wall", "wall"])
    sim = M.Simulation(cfg)
    with pytest.raises(M.MPMError) as e:
        sim.set_obstacle_profile([np.array([[0.1, 0.2], [0.1, 0.2]])])
    assert e.value.status == "MPM_EINVAL"
    with pytest.raises(M.MPMError) as e:      # obstacle on the inflow face
        sim.set_obstacle_profile([_square((0.02, 0.25), 0.05, 0.0)])
    assert e.value.status == "MPM_EINVAL"
    with pytest.raises(M.MPMError) as e:
        sim.set_obstacle_profile([np.array([[0.5, 0.6, np.nan], [0.2, 0.2, 0.3]])])
    assert e.value.status == "MPM_EINVAL"
    sim.close()
    sim3 = M.Simulation(I.base_config(3, [16, 16, 16], 1 / 16, ["wall"] * 6))
    with pytest.raises(M.MPMError) as e:
        sim3.set_obstacle_profile([_square((0.5, 0.5), 0.1, 0.0)])
    assert e.value.status == "MPM_EUNSUPPORTED"
    sim3.close()


def _compare(g, o, dim, tol):
    ig, io = np.argsort(g.read("ID")), np.argsort(o.read("ID"))
    for f in ("RHO", "P", "E"):
        a, b = g.read(f)[ig], o.read(f)[io]
        assert np.abs(a - b).sum() / np.abs(b).sum() <= tol, f
    va, vb = g.read("V")[:, ig], o.read("V")[:, io]
    assert np.abs(va - vb).sum() / np.abs(vb).sum() <= tol


@pytest.mark.parametrize("precision,steps,tol", [("fp64", 40, 1e-9), ("fp32", 100, 1e-4)])
def test_flow_past_a_profile_matches_the_oracle(precision, steps, tol):
    p = I.aerofoil(nx=120, ny=81, ppa=2, precision=precision)
    if precision == "fp32":
        for k in ("x", "v", "mass", "rho", "e"):
            setattr(p, k, getattr(p, k).astype(np.float32).astype(np.float64))
    g = M.Simulation.from_problem(p)
    o = O.OracleSim(p.cfg)
    o.add_particles(p.x, p.v, p.mass, p.rho, p.e)
    om, on, _ = O.obstacle_profile(p.cfg, p.profile)
    o.set_obstacle_mask(om, on)
    g.step(steps)
    o.step(steps)
    _compare(g, o, 2, tol)
    g.close()


def test_aerofoil_flow_is_faster_over_the_upper_surface():
    """The aerofoil case (Sec. 4.1, Fig. oat15a): at 25 degrees the flow speeds up
    approaching the profile, more over the upper surface than under it.  Mean
    particle speed in bands along 10-90% of the chord, up to 0.11 chords from
    the chord line, after t = 0.3 (about two chord passages)."""
    p = I.aerofoil(nx=300, ny=203, ppa=2)
    le, chord, ang = np.array([0.1, 0.15]), 0.1, np.deg2rad(25.0)
    tdir = np.array([np.cos(-ang), np.sin(-ang)])
    ndir = np.array([-tdir[1], tdir[0]])
    with M.Simulation.from_problem(p) as s:
        s.step(1000000, t_end=0.3)
        x, v = s.read("X"), s.read("V")
    rel = x - le[:, None]
    along, up = rel.T @ tdir, rel.T @ ndir
    speed = np.sqrt((v ** 2).sum(axis=0))
    band = (along > 0.1 * chord) & (along < 0.9 * chord) & (np.abs(up) < 0.11 * chord)
    above, below = speed[band & (up > 0)].mean(), speed[band & (up < 0)].mean()
    assert above > 1.2 * below and below > 0.73, (above, below)
