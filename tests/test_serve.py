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
