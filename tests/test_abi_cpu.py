"""CPU-only checks of the boundary: the CUDA library builds for sm_103a,
loads, and exports every entry point include/mpm.h declares; the Python
binding names the same entry points.  No compute call is made here."""
import ctypes
import os
import re

from paper_2404_17057_b300 import build as B
from paper_2404_17057_b300 import mpm as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "mpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    assert sorted(M.EXPORTS) == declared()
    L = M.load()
    for n in M.EXPORTS:
        assert hasattr(L, n)


def test_library_is_built_for_sm_103a():
    cmd = " ".join(B.ARCH)
    assert "sm_103a" in cmd and "compute_103a" in cmd


def test_null_handles_are_rejected_without_a_device():
    L = M.load()
    assert L.mpm_field_size(None, 0) == -1
    assert L.mpm_sync(None) == 1
    assert L.mpm_step(None, 1, 0.0, 0.0) == 1
    assert L.mpm_create(None, None) == 1
    L.mpm_destroy(None)
    assert L.mpm_batch_create(None, None) == 1
    assert L.mpm_batch_add(None, None, 1, 0.0, 0.0) == 1
    assert L.mpm_batch_remove(None, None) == 1
    assert L.mpm_batch_step_async(None, 1) == 1
    assert L.mpm_batch_sync(None) == 1
    L.mpm_batch_destroy(None)
    assert L.mpm_check_fixed_rounding(None, None) == 1
    assert L.mpm_set_obstacle_profile(None, 1, None, None, None, None, None) == 1


def test_coloured_mode_rejects_overlapping_colour_windows_without_a_device():
    # configuration checks run before any CUDA call
    from paper_2404_17057_b300 import inputs as I
    L = M.load()
    bad = [
        # tile edge 1 < degree 2: same-colour windows would meet
        I.base_config(3, [32, 32, 32], 1 / 32, ["wall"] * 6, precision="fp32_coloured", tile=[32, 8, 1]),
        # periodic axis of 40 cells is not a whole number of 32-span tiles
        I.base_config(2, [40, 16], 1 / 40, ["periodic"] * 4, precision="fp32_coloured", tile=[32, 8, 1]),
        # periodic axis of one tile: the window wraps onto itself
        I.base_config(2, [32, 16], 1 / 32, ["periodic"] * 4, precision="fp32_coloured", tile=[32, 8, 1]),
    ]
    for cfg in bad:
        h = ctypes.c_void_p()
        assert L.mpm_create(ctypes.byref(M.make_config(cfg)), ctypes.byref(h)) == 7
        assert not h.value
    bad_prec = I.base_config(2, [64, 16], 1 / 64, ["wall"] * 4, precision=4)
    assert L.mpm_create(ctypes.byref(M.make_config(bad_prec)), ctypes.byref(ctypes.c_void_p())) == 1
