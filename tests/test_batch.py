"""Batched execution (mpm_batch_*): many simulations, one launch per stage.

Every member runs the same tile code as alone, so fixed-point members agree
with their solo runs bit for bit and FP32 members (float atomics, whose
order varies between launches) to the FP32 rounding level.  Members of
different kernel variants share a batch; budgets that end inside a chunk
leave a member idle, not advanced; the membership rules are enforced."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2404_17057_b300 import inputs as I
from paper_2404_17057_b300 import mpm as M

pytestmark = pytest.mark.gpu


def solo(prob, steps):
    s = M.Simulation.from_problem(prob)
    s.step(steps)
    out = state(s)
    s.close()
    return out


def state(s):
    ids = s.read("ID").astype(np.int64)
    o = np.argsort(ids)
    return {f: s.read(f)[..., o] for f in ("X", "V", "RHO", "E", "Q")} | {"clock": s.read("CLOCK"),
                                                                         "cons": s.conservation()}


def problems(precision):
    a = I.shock_tube(ncell=96, ny=4, precision=precision)
    b = I.request_problem({"kind": "cylinder", "side": 128, "steps": 30, "precision": precision,
                           "radius": 0.06, "mach": 2.5, "seed": 11})
    c = I.request_problem({"kind": "shock_tube", "side": 160, "steps": 30, "precision": precision})
    d = I.blast(n=16, precision=precision)
    return [a, b, c, d]


# fp64: the batched 2D members run the span kernels, alone the small grids
# run the generic ones; the sums differ in order only
@pytest.mark.parametrize("precision", ["fp32_fixed64", "fp32", "fp64"])
def test_batch_equals_alone(precision):
    probs = problems(precision)
    budgets = [23, 30, 17, 30]                 # not multiples of the chunk: members idle inside a chunk
    ref = [solo(p, n) for p, n in zip(probs, budgets)]
    sims = [M.Simulation.from_problem(p) for p in probs]
    b = M.Batch()
    for s, n in zip(sims, budgets):
        b.add(s, n)
    for _ in range(3):
        b.step_async(10)
    b.sync()
    info = b.info()
    assert info["members"] == 4 and info["groups"] >= 3 and info["recordings"] == 1
    for s in sims:
        b.remove(s)
    b.close()
    for s, r, n in zip(sims, ref, budgets):
        got = state(s)
        assert int(got["clock"][2]) == n
        for f in ("X", "V", "RHO", "E", "Q", "clock", "cons"):
            if precision == "fp32_fixed64":
                assert np.array_equal(got[f], r[f]), f
            else:
                scale = np.abs(r[f]).max() + 1e-30
                tol = 1e-11 if precision == "fp64" else 1e-5
                assert np.abs(got[f] - r[f]).max() <= tol * scale, f
        s.close()


def test_members_join_and_leave_between_chunks():
    probs = problems("fp32_fixed64")
    ref = [solo(p, 20) for p in probs]
    sims = [M.Simulation.from_problem(p) for p in probs]
    b = M.Batch()
    b.add(sims[0], 20)
    b.add(sims[1], 20)
    b.step_async(8)
    b.add(sims[2], 20)                         # joins late
    b.step_async(8)
    b.remove(sims[0])                          # leaves before its budget ends
    b.add(sims[3], 20)
    b.step_async(12)
    b.sync()
    sims[0].step(4)                            # continues alone after leaving
    for s in sims[1:]:
        b.remove(s)                            # 20, 20 and 12 steps done
    b.add(sims[3], 8)                          # rejoins alone for part of the rest
    b.step_async(5)
    b.sync()
    b.remove(sims[3])
    sims[3].step(3)
    assert b.info()["recordings"] == 4
    b.close()
    for s, r in zip(sims, ref):
        got = state(s)
        assert int(got["clock"][2]) == 20
        for f in ("X", "V", "RHO", "E", "Q", "cons"):
            assert np.array_equal(got[f], r[f]), f
        s.close()


def test_membership_rules():
    p = I.shock_tube(ncell=64, ny=4, precision="fp32_fixed64")
    s = M.Simulation.from_problem(p)
    b = M.Batch()
    b.add(s, 5)
    with pytest.raises(M.MPMError) as e:
        s.step(1)
    assert e.value.status == "MPM_ESTATE"
    with pytest.raises(M.MPMError) as e:
        s.read("RHO")
    assert e.value.status == "MPM_ESTATE"
    with pytest.raises(M.MPMError) as e:
        b.add(s, 5)                            # already a member
    assert e.value.status == "MPM_ESTATE"
    other = M.Simulation.from_problem(p)
    with pytest.raises(M.MPMError) as e:
        M.mpm_batch_add(b._h, other.handle, 0)  # a budget is required
    assert e.value.status == "MPM_EINVAL"
    other.close()
    b.step_async(3)
    b.remove(s)
    s.step(1)
    assert int(s.read("CLOCK")[2]) == 4
    b.add(s, 2)
    s.close()                                  # destroying a member leaves the batch first
    b.members.clear()
    assert b.info()["members"] == 0
    b.step_async(1)                            # empty batch: nothing to do
    b.close()


def test_tile_tuner_picks_a_valid_shape_once():
    from paper_2404_17057_b300 import tune as T
    p = I.request_problem({"kind": "cylinder", "side": 128, "steps": 10, "precision": "fp32_fixed64",
                           "radius": 0.05, "mach": 3.0, "seed": 3})
    t = T.TileTuner(steps=2, warmup=1)
    tile = t.tile_for(p)
    assert tuple(tile) in T.CANDIDATES[2]
    key = t.problem_class(p)
    assert min(v for v in t.timings[key].values() if v is not None) > 0
    assert t.tile_for(p) == tile and len(t.timings) == 1
    q = I.request_problem({"kind": "cylinder", "side": 128, "steps": 10, "precision": "fp32_fixed64",
                           "radius": 0.05, "mach": 3.0, "seed": 3})
    q.cfg["tile"] = tile
    a = solo(q, 10)
    q.cfg["tile"] = [0, 0, 0]
    d = solo(q, 10)
    # the tile changes the work split, not the result (fixed-point sums)
    for f in ("RHO", "E", "V"):
        assert np.array_equal(a[f], d[f]), f
