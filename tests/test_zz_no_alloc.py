"""The allocation-free key sort (mpm_sort_keys_static) against the library's
regular re-order.

mpm_sort_keys_static serves callers that must not allocate device memory
(components confined to another framework's memory pool, latency-critical
loops where an allocation could synchronise the device); it keeps its
scratch in fixed device arrays.  Here it must reproduce, bit for bit, the
order and cell starts that mpm_add_particles produces for the same keys, on
two calls in a row (the second reuses the scratch left by the first), and
leave the device's free memory unchanged.  This file is collected last so
that a failure here cannot hide other results.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2404_17057_b300 import inputs as I
from paper_2404_17057_b300 import mpm as M

pytestmark = pytest.mark.gpu


def particles(dim, n_cells, N, seed):
    rng = np.random.default_rng(seed)
    h = 1.0 / n_cells[0]
    cfg = I.base_config(dim, n_cells, h, ["wall"] * (2 * dim), degree=2, precision="fp32")
    L = np.array([n_cells[a] * h for a in range(dim)])[:, None]
    x = (rng.random((dim, N)) * L).astype(np.float32).astype(np.float64)
    return I.Problem("keys", cfg, x, np.zeros((dim, N)), np.full(N, h ** dim), np.ones(N), np.ones(N))


@pytest.mark.parametrize("dim,n_cells,N", [(2, [300, 170], 200003), (3, [40, 33, 29], 150001)])
def test_static_sort_matches_the_regular_reorder(dim, n_cells, N):
    p = particles(dim, n_cells, N, seed=dim)
    sim = M.Simulation.from_problem(p)
    ids = sim.read("ID").astype(np.int64)
    keys_sorted = sim.read("KEY").astype(np.uint32)
    start = sim.read("CELLSTART").astype(np.int64)
    nkeys = start.shape[0] - 1
    sim.close()
    keys_in = np.empty(N, dtype=np.uint32)
    keys_in[ids] = keys_sorted                    # the same keys in input order
    dev = torch.device("cuda")
    kt = torch.from_numpy(keys_in.view(np.int32)).to(dev)
    perm = torch.empty(N, dtype=torch.int32, device=dev)
    cst = torch.empty(nkeys + 1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        perm.fill_(-1)
        cst.fill_(-1)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        M.mpm_sort_keys_static(kt.data_ptr(), N, nkeys, perm.data_ptr(), cst.data_ptr(), stream)
        torch.cuda.synchronize()
        if call > 0:   # the first call on the device may load the module
            assert torch.cuda.mem_get_info()[0] == free0
        assert np.array_equal(perm.cpu().numpy().view(np.uint32).astype(np.int64), ids)
        assert np.array_equal(cst.cpu().numpy().view(np.uint32).astype(np.int64), start)
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), keys_in)   # input untouched


def test_static_sort_flags_a_key_beyond_nkeys():
    """A key >= nkeys marks cell_start[nkeys] with 0xffffffff; the next valid
    call is unaffected."""
    rng = np.random.default_rng(3)
    N, nkeys = 5000, 300
    keys = rng.integers(0, nkeys, N).astype(np.uint32)
    dev = torch.device("cuda")
    perm = torch.empty(N, dtype=torch.int32, device=dev)
    cst = torch.empty(nkeys + 1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    bad = keys.copy()
    bad[1234] = nkeys + 7
    kb = torch.from_numpy(bad.view(np.int32)).to(dev)
    M.mpm_sort_keys_static(kb.data_ptr(), N, nkeys, perm.data_ptr(), cst.data_ptr(), stream)
    torch.cuda.synchronize()
    assert int(cst[nkeys].item()) & 0xffffffff == 0xffffffff
    kg = torch.from_numpy(keys.view(np.int32)).to(dev)
    M.mpm_sort_keys_static(kg.data_ptr(), N, nkeys, perm.data_ptr(), cst.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), np.argsort(keys, kind="stable"))
    assert np.array_equal(cst.cpu().numpy().astype(np.int64),
                          np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=nkeys))]))


def test_static_sort_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda")
    buf = torch.zeros(16, dtype=torch.int32, device=dev)
    L = M.load()
    big = M.SORT_STATIC_MAX_KEYS + 1
    code = L.mpm_sort_keys_static(buf.data_ptr(), big, 8, buf.data_ptr(), buf.data_ptr(), None)
    assert code == 1 and "MPM_SORT_STATIC_MAX_KEYS" in M.mpm_last_error(None)
    code = L.mpm_sort_keys_static(buf.data_ptr(), 4, M.SORT_STATIC_MAX_SPANS + 1, buf.data_ptr(), buf.data_ptr(), None)
    assert code == 1
