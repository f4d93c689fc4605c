"""Serving: continuous batching over independent problems.

GPU: every result produced in the mix equals the same request solved alone
(bit for bit in the fixed-point mode, whose P2G sums are order independent),
problems are resident concurrently, and the loop reports latency.
CPU: the request stream is seeded and has the requested distribution."""
import numpy as np
import pytest

from paper_2404_17057_b300 import inputs as I


def test_request_stream_is_seeded_and_well_formed():
    a = I.serving_stream(count=200, seed=5)
    b = I.serving_stream(count=200, seed=5)
    assert a == b
    kinds = {r["kind"] for r in a}
    assert kinds == {"shock_tube", "cylinder"}
    sides = np.array([r["side"] for r in a])
    assert sides.min() >= 64 and sides.max() <= 1024 and np.all(sides % 16 == 0)
    arr = np.array([r["arrival"] for r in a])
    assert np.all(np.diff(arr) > 0)
    rate = len(a) / arr[-1]
    assert 35 < rate < 70                      # Poisson arrivals at 50/s
    for r in a:
        if r["kind"] == "cylinder":
            assert 0.02 <= r["radius"] <= 0.1 and 1.5 <= r["mach"] <= 4.0


@pytest.mark.gpu
def test_mix_equals_alone_bit_for_bit():
    pytest.importorskip("torch")
    from paper_2404_17057_b300 import serve as S
    reqs = I.serving_stream(count=10, seed=7, steps=40, side_lo=64, side_hi=160)
    mixed, stats = S.Server(chunk=10).run(reqs, realtime=False)
    alone, _ = S.run_sequential(reqs, realtime=False)
    assert len(mixed) == len(alone) == len(reqs)
    a = {r.rid: r for r in alone}
    for r in mixed:
        b = a[r.rid]
        assert np.array_equal(r.rho[np.argsort(r.ids)], b.rho[np.argsort(b.ids)])
        assert np.array_equal(r.conservation, b.conservation)
    assert stats["p99_s"] >= stats["p50_s"] > 0


@pytest.mark.gpu
def test_a_failing_request_is_retired_and_the_others_finish():
    """A request whose time step violates the method's CFL rule (one span per
    step) fails with MPM_ECFL in the mix; the server retires it with that
    error and the other requests still equal their solo runs."""
    pytest.importorskip("torch")
    from paper_2404_17057_b300 import serve as S
    reqs = I.serving_stream(count=4, seed=11, steps=30, side_lo=64, side_hi=128)
    reqs[1] = dict(reqs[1], cfl=5.0)
    mixed, stats = S.Server(chunk=7).run(reqs, realtime=False)
    alone, _ = S.run_sequential(reqs, realtime=False)
    m = {r.rid: r for r in mixed}
    a = {r.rid: r for r in alone}
    assert m[reqs[1]["id"]].error == "MPM_ECFL" == a[reqs[1]["id"]].error
    assert stats["failed"] == 1 and stats["solves"] == 3
    for r in reqs:
        if r["id"] == reqs[1]["id"]:
            continue
        x, y = m[r["id"]], a[r["id"]]
        assert not x.error and np.array_equal(x.rho[np.argsort(x.ids)], y.rho[np.argsort(y.ids)])


def test_serving_problems_use_normalised_fixed_point_units():
    reqs = I.serving_stream(count=6, seed=3, steps=10, side_lo=64, side_hi=128)
    for r in reqs:
        p = I.request_problem(r)
        um, umom, uf = p.cfg["fixed_unit"]
        assert um == pytest.approx(I.MASS_UNIT_PER_PARTICLE * float(np.mean(p.mass)))
        assert umom > um > 0 and uf > umom
