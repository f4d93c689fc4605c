"""Multi-GPU host logic on CPU: the benchmark runs independent replicas, one
per rank (no data-path collective); the job time is the slowest rank's and
the job value counts every rank's particles.  Two gloo ranks stand in for two
GPUs.  The reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    v = bench.job_value(1000, 20, world, ms)
    dist.barrier()
    q.put((rank, ms, v))
    dist.destroy_process_group()


def test_replicas_time_is_the_slowest_rank_and_value_counts_all_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, v in res:
        assert ms == 15.0
        assert v == pytest.approx(1000 * 20 * 2 / 0.015)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.job_value(10, 3, 1, 1.0) == pytest.approx(30000.0)


def test_reference_arm_prints_nothing_on_other_ranks(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    args = bench.parse()
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(args)
    assert out.getvalue() == ""
