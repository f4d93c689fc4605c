"""Python binding of the C ABI in include/mpm.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments; all work happens in ``libmpm.so``.  Device
memory comes from PyTorch's caching allocator (through the ABI's alloc hook)
and the simulation runs on PyTorch's current CUDA stream unless told
otherwise.  There is no CPU fallback: without the compiled library or a CUDA
device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmpm.so")

BC = {"wall": 0, "periodic": 1, "inflow": 2, "outflow": 3}
PRECISION = {"fp32": 0, "fp32_fixed64": 1, "fp64": 2, "fp32_coloured": 3}
FIELDS = {"X": 0, "V": 1, "M": 2, "RHO": 3, "E": 4, "P": 5, "Q": 6, "ID": 7, "KEY": 8,
          "CELLSTART": 9, "GRID_M": 10, "GRID_MV": 11, "GRID_F": 12, "GRID_MV2": 13, "CLOCK": 14,
          "GEN": 16}
STATUS = {0: "MPM_OK", 1: "MPM_EINVAL", 2: "MPM_ENOMEM", 3: "MPM_ECUDA", 4: "MPM_ESTATE",
          5: "MPM_ENONFINITE", 6: "MPM_ETIMEOUT", 7: "MPM_EUNSUPPORTED", 8: "MPM_ECFL"}

EXPORTS = ["mpm_create", "mpm_add_particles", "mpm_add_particles_f32", "mpm_set_obstacle_mask", "mpm_set_obstacle_profile",
           "mpm_cfl_dt", "mpm_step", "mpm_step_async", "mpm_sync", "mpm_read_state", "mpm_read_grid_fixed",
           "mpm_field_size", "mpm_conservation", "mpm_sizes", "mpm_profile", "mpm_profile_read", "mpm_stream",
           "mpm_last_error", "mpm_destroy", "mpm_sort_keys_static", "mpm_check_fixed_rounding",
           "mpm_batch_create", "mpm_batch_add", "mpm_batch_remove", "mpm_batch_step_async", "mpm_batch_sync",
           "mpm_batch_info", "mpm_batch_stream", "mpm_batch_last_error", "mpm_batch_destroy"]
SORT_STATIC_MAX_KEYS = 262144
SORT_STATIC_MAX_SPANS = 16777216


class MPMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class mpm_config(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double), ("origin", C.c_double * 3),
                ("gamma", C.c_double), ("c0", C.c_double), ("c1", C.c_double), ("degree", C.c_int),
                ("precision", C.c_int), ("fixed_unit", C.c_double * 3), ("bc", C.c_int * 6),
                ("inflow_rho", C.c_double), ("inflow_p", C.c_double), ("inflow_v", C.c_double * 3),
                ("cfl", C.c_double), ("sort_interval", C.c_int), ("seed", C.c_uint64), ("tile", C.c_int * 3),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libmpm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2404_17057_b300.build.build()")
    L = C.CDLL(path)
    P, vp, i64, d = C.POINTER, C.c_void_p, C.c_int64, C.c_double
    L.mpm_create.argtypes = [P(mpm_config), P(vp)]
    L.mpm_add_particles.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.mpm_add_particles_f32.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.mpm_set_obstacle_mask.argtypes = [vp, vp, vp]
    L.mpm_set_obstacle_profile.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.mpm_cfl_dt.argtypes = [vp, P(d)]
    L.mpm_step.argtypes = [vp, i64, d, d]
    L.mpm_step_async.argtypes = [vp, i64, d, d]
    L.mpm_sync.argtypes = [vp]
    L.mpm_read_state.argtypes = [vp, C.c_int, vp, i64]
    L.mpm_read_grid_fixed.argtypes = [vp, C.c_int, vp, i64]
    L.mpm_field_size.argtypes = [vp, C.c_int]
    L.mpm_field_size.restype = i64
    L.mpm_conservation.argtypes = [vp, vp]
    L.mpm_sizes.argtypes = [vp, vp]
    L.mpm_profile.argtypes = [vp, C.c_int]
    L.mpm_profile_read.argtypes = [vp, vp, vp, C.c_int]
    L.mpm_stream.argtypes = [vp]
    L.mpm_stream.restype = vp
    L.mpm_last_error.argtypes = [vp]
    L.mpm_last_error.restype = C.c_char_p
    L.mpm_destroy.argtypes = [vp]
    L.mpm_destroy.restype = None
    L.mpm_sort_keys_static.argtypes = [vp, i64, i64, vp, vp, vp]
    L.mpm_check_fixed_rounding.argtypes = [P(C.c_uint64), P(C.c_uint32)]
    L.mpm_batch_create.argtypes = [vp, P(vp)]
    L.mpm_batch_add.argtypes = [vp, vp, i64, d, d]
    L.mpm_batch_remove.argtypes = [vp, vp]
    L.mpm_batch_step_async.argtypes = [vp, i64]
    L.mpm_batch_sync.argtypes = [vp]
    L.mpm_batch_info.argtypes = [vp, vp]
    L.mpm_batch_stream.argtypes = [vp]
    L.mpm_batch_stream.restype = vp
    L.mpm_batch_last_error.argtypes = [vp]
    L.mpm_batch_last_error.restype = C.c_char_p
    L.mpm_batch_destroy.argtypes = [vp]
    L.mpm_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("mpm_field_size", "mpm_stream", "mpm_last_error", "mpm_destroy", "mpm_batch_stream",
                        "mpm_batch_last_error", "mpm_batch_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(code: int, handle=None):
    if code != 0:
        msg = load().mpm_last_error(handle)
        raise MPMError(code, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator on a given stream."""

    def __init__(self, stream_ptr):
        import torch
        self.torch = torch
        self.stream = stream_ptr
        self.device = torch.cuda.current_device()
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return int(self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:       # out of memory -> the library reports MPM_ENOMEM
            return None

    def _free(self, ptr, ctx):
        self.torch.cuda.caching_allocator_delete(int(ptr))


def make_config(cfg: dict, stream=None, allocator=None) -> mpm_config:
    c = mpm_config()
    c.dim = int(cfg["dim"])
    n = list(cfg["n"]) + [1] * (3 - len(cfg["n"]))
    c.n = (C.c_int * 3)(*[int(v) for v in n[:3]])
    c.h = float(cfg["h"])
    o = list(cfg.get("origin", [0.0] * 3)) + [0.0] * 3
    c.origin = (C.c_double * 3)(*[float(v) for v in o[:3]])
    c.gamma = float(cfg.get("gamma", 1.4))
    c.c0 = float(cfg.get("c0", 1.0))
    c.c1 = float(cfg.get("c1", 1.0))
    c.degree = int(cfg.get("degree", 2))
    prec = cfg.get("precision", "fp32")
    c.precision = PRECISION[prec] if isinstance(prec, str) else int(prec)
    fu = list(cfg.get("fixed_unit", [0.0] * 3)) + [0.0] * 3
    c.fixed_unit = (C.c_double * 3)(*[float(v) for v in fu[:3]])
    bc = [BC[b] if isinstance(b, str) else int(b) for b in cfg["bc"]] + [0] * 6
    c.bc = (C.c_int * 6)(*bc[:6])
    c.inflow_rho = float(cfg.get("inflow_rho", 1.0))
    c.inflow_p = float(cfg.get("inflow_p", 1.0))
    iv = list(cfg.get("inflow_v", [0.0] * 3)) + [0.0] * 3
    c.inflow_v = (C.c_double * 3)(*[float(v) for v in iv[:3]])
    c.cfl = float(cfg.get("cfl", 0.4))
    c.sort_interval = int(cfg.get("sort_interval", 1))
    c.seed = int(cfg.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    t = list(cfg.get("tile", [0, 0, 0])) + [0, 0, 0]
    c.tile = (C.c_int * 3)(*[int(v) for v in t[:3]])
    c.stream = stream
    if allocator is not None:
        c.alloc = allocator.alloc
        c.free = allocator.free
    return c


# ----------------------------------------------------------- the ABI calls

def mpm_create(cfg: dict, stream=None, torch_memory: bool = True):
    """Returns (handle, keepalive); keepalive must outlive the handle."""
    L = load()
    alloc = None
    if torch_memory:
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the MPM library has no CPU path")
        own = None
        if stream is None:
            own = torch.cuda.Stream()           # one stream per simulation
            stream = own.cuda_stream
        alloc = _TorchAllocator(stream)
        alloc.owned_stream = own
    c = make_config(cfg, stream=stream, allocator=alloc)
    h = C.c_void_p()
    code = L.mpm_create(C.byref(c), C.byref(h))
    if code != 0:
        msg = L.mpm_last_error(None)
        raise MPMError(code, msg.decode() if msg else "")
    return h, (c, alloc)


def mpm_add_particles(h, x, v, mass, rho, e):
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    mass, rho, e = (np.ascontiguousarray(a, dtype=np.float64) for a in (mass, rho, e))
    _check(load().mpm_add_particles(h, int(mass.shape[0]), _ptr(x), _ptr(v), _ptr(mass), _ptr(rho), _ptr(e)), h)


def mpm_add_particles_f32(h, x, v, mass, rho, e):
    x = np.ascontiguousarray(x, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    mass, rho, e = (np.ascontiguousarray(a, dtype=np.float32) for a in (mass, rho, e))
    _check(load().mpm_add_particles_f32(h, int(mass.shape[0]), _ptr(x), _ptr(v), _ptr(mass), _ptr(rho), _ptr(e)), h)


def mpm_set_obstacle_mask(h, mask, normals):
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    normals = np.ascontiguousarray(normals, dtype=np.float64)
    _check(load().mpm_set_obstacle_mask(h, _ptr(mask), _ptr(normals)), h)


def mpm_cfl_dt(h) -> float:
    out = C.c_double()
    _check(load().mpm_cfl_dt(h, C.byref(out)), h)
    return out.value


def mpm_step(h, nsteps: int, dt: float = 0.0, t_end: float = 0.0):
    _check(load().mpm_step(h, int(nsteps), float(dt), float(t_end)), h)


def mpm_step_async(h, nsteps: int, dt: float = 0.0, t_end: float = 0.0):
    _check(load().mpm_step_async(h, int(nsteps), float(dt), float(t_end)), h)


def mpm_sync(h):
    _check(load().mpm_sync(h), h)


def mpm_field_size(h, field) -> int:
    f = FIELDS[field] if isinstance(field, str) else int(field)
    return int(load().mpm_field_size(h, f))


def mpm_read_state(h, field, dim: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    f = FIELDS[field] if isinstance(field, str) else int(field)
    n = mpm_field_size(h, f)
    if out is None:
        out = np.empty(max(n, 0), dtype=np.float64)
    elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size < n:
        raise ValueError("out must be a contiguous float64 array of the field's size")
    out = out.reshape(-1)[:max(n, 0)]
    _check(load().mpm_read_state(h, f, _ptr(out), n), h)
    if dim and field in ("X", "V", "GRID_MV", "GRID_F", "GRID_MV2"):
        out = out.reshape(dim, -1)
    return out


def mpm_read_grid_fixed(h, field, dim: int | None = None) -> np.ndarray:
    f = FIELDS[field] if isinstance(field, str) else int(field)
    n = mpm_field_size(h, f)
    out = np.empty(n, dtype=np.int64)
    _check(load().mpm_read_grid_fixed(h, f, _ptr(out), n), h)
    if dim and field != "GRID_M":
        out = out.reshape(dim, -1)
    return out


def mpm_set_obstacle_profile(h, loops):
    loops = [np.asarray(l, dtype=np.float64) for l in loops]
    lens = np.ascontiguousarray([l.shape[1] for l in loops], dtype=np.int64)
    pts = np.ascontiguousarray(np.concatenate(loops, axis=1))
    nn = mpm_field_size(h, FIELDS["GRID_M"])
    mask = np.empty(nn, dtype=np.uint8)
    nrm = np.empty(2 * nn)
    sd = np.empty(nn)
    _check(load().mpm_set_obstacle_profile(h, len(loops), _ptr(lens), _ptr(pts), _ptr(mask), _ptr(nrm), _ptr(sd)),
           h)
    return mask, nrm.reshape(2, nn), sd


def mpm_conservation(h) -> np.ndarray:
    out = np.empty(5, dtype=np.float64)
    _check(load().mpm_conservation(h, _ptr(out)), h)
    return out


def mpm_sizes(h) -> dict:
    out = np.empty(4, dtype=np.int64)
    _check(load().mpm_sizes(h, _ptr(out)), h)
    return {"particles": int(out[0]), "nodes": int(out[1]), "keys": int(out[2]), "steps": int(out[3])}


def mpm_profile(h, enable: bool):
    _check(load().mpm_profile(h, int(bool(enable))), h)


def mpm_profile_read(h, reset: bool = False):
    ms = np.zeros(8, dtype=np.float64)
    cnt = np.zeros(8, dtype=np.int64)
    _check(load().mpm_profile_read(h, _ptr(ms), _ptr(cnt), int(bool(reset))), h)
    return ms, cnt


def mpm_stream(h) -> int:
    return int(load().mpm_stream(h) or 0)


def mpm_last_error(h=None) -> str:
    m = load().mpm_last_error(h)
    return m.decode() if m else ""


def mpm_destroy(h):
    load().mpm_destroy(h)


def mpm_sort_keys_static(keys_ptr: int, n: int, nkeys: int, perm_ptr: int, cell_start_ptr: int, stream: int = 0):
    """Allocation-free stable key sort on caller device buffers (raw pointers).

    For callers that must not allocate device memory (graph capture, a
    foreign memory pool, latency-critical loops).  n is capped at
    SORT_STATIC_MAX_KEYS; concurrent calls on one device must not overlap."""
    _check(load().mpm_sort_keys_static(keys_ptr, int(n), int(nkeys), perm_ptr, cell_start_ptr, stream or None))


def mpm_check_fixed_rounding() -> tuple[int, int]:
    """(mismatches, first mismatching bit pattern) of the fixed-point
    quantiser's 32-bit rounding against the float-to-int64 conversion over
    every binary32 input below 2^31 in magnitude; (0, 0xffffffff) when they
    agree everywhere."""
    bad, first = C.c_uint64(0), C.c_uint32(0)
    _check(load().mpm_check_fixed_rounding(C.byref(bad), C.byref(first)))
    return int(bad.value), int(first.value)


def _bcheck(code: int, bh=None):
    if code != 0:
        msg = load().mpm_batch_last_error(bh)
        raise MPMError(code, msg.decode() if msg else "")


def mpm_batch_create(stream=None):
    h = C.c_void_p()
    _bcheck(load().mpm_batch_create(stream, C.byref(h)))
    return h


def mpm_batch_add(bh, h, nsteps: int, dt: float = 0.0, t_end: float = 0.0):
    _bcheck(load().mpm_batch_add(bh, h, int(nsteps), float(dt), float(t_end)), bh)


def mpm_batch_remove(bh, h):
    _bcheck(load().mpm_batch_remove(bh, h), bh)


def mpm_batch_step_async(bh, nsteps: int):
    _bcheck(load().mpm_batch_step_async(bh, int(nsteps)), bh)


def mpm_batch_sync(bh):
    _bcheck(load().mpm_batch_sync(bh), bh)


def mpm_batch_info(bh) -> dict:
    out = np.zeros(4, dtype=np.int64)
    _bcheck(load().mpm_batch_info(bh, _ptr(out)), bh)
    return {"members": int(out[0]), "groups": int(out[1]), "launches_per_step": int(out[2]),
            "recordings": int(out[3])}


def mpm_batch_stream(bh) -> int:
    return int(load().mpm_batch_stream(bh) or 0)


def mpm_batch_destroy(bh):
    load().mpm_batch_destroy(bh)


# ------------------------------------------------------------ convenience

class Simulation:
    """Owning wrapper of one mpm_sim handle."""

    def __init__(self, cfg: dict, stream=None, torch_memory: bool = True):
        self.cfg = dict(cfg)
        self.dim = int(cfg["dim"])
        self._h, self._keep = mpm_create(cfg, stream=stream, torch_memory=torch_memory)

    @classmethod
    def from_problem(cls, prob, f32=False, **kw):
        """f32: upload the initial state as binary32 (mpm_add_particles_f32)."""
        s = cls(prob.cfg, **kw)
        if f32:
            s.add_particles_f32(prob.x, prob.v, prob.mass, prob.rho, prob.e)
        else:
            s.add_particles(prob.x, prob.v, prob.mass, prob.rho, prob.e)
        if prob.mask is not None:
            s.set_obstacle_mask(prob.mask, prob.normals)
        if getattr(prob, "profile", None):
            s.set_obstacle_profile(prob.profile)
        return s

    @property
    def handle(self):
        return self._h

    def add_particles(self, x, v, mass, rho, e):
        mpm_add_particles(self._h, x, v, mass, rho, e)

    def add_particles_f32(self, x, v, mass, rho, e):
        mpm_add_particles_f32(self._h, x, v, mass, rho, e)

    def set_obstacle_mask(self, mask, normals):
        mpm_set_obstacle_mask(self._h, mask, normals)

    def set_obstacle_profile(self, loops):
        """Obstacle from closed loops of boundary points, each (2, k); returns
        the installed mask, normals (2, nodes) and the signed distance."""
        return mpm_set_obstacle_profile(self._h, loops)

    def cfl_dt(self) -> float:
        return mpm_cfl_dt(self._h)

    def step(self, nsteps: int, dt: float = 0.0, t_end: float = 0.0):
        mpm_step(self._h, nsteps, dt, t_end)

    def step_async(self, nsteps: int, dt: float = 0.0, t_end: float = 0.0):
        mpm_step_async(self._h, nsteps, dt, t_end)

    def sync(self):
        mpm_sync(self._h)

    def read(self, field: str, out: np.ndarray | None = None) -> np.ndarray:
        """Field values as float64; `out` (optional) receives them, e.g. a
        page-locked array for a faster device-to-host copy."""
        return mpm_read_state(self._h, field, self.dim, out)

    def read_fixed(self, field: str) -> np.ndarray:
        return mpm_read_grid_fixed(self._h, field, self.dim)

    def conservation(self) -> np.ndarray:
        return mpm_conservation(self._h)

    def sizes(self) -> dict:
        return mpm_sizes(self._h)

    def profile(self, enable: bool):
        mpm_profile(self._h, enable)

    def profile_read(self, reset: bool = False):
        return mpm_profile_read(self._h, reset)

    @property
    def stream(self) -> int:
        return mpm_stream(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None:
            mpm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Owning wrapper of one mpm_batch handle (members are Simulation objects)."""

    def __init__(self, stream=None):
        import torch
        self._own = None
        if stream is None:
            self._own = torch.cuda.Stream()
            stream = self._own.cuda_stream
        self._h = mpm_batch_create(stream)
        self.members: list[Simulation] = []

    def add(self, sim: Simulation, nsteps: int, dt: float = 0.0, t_end: float = 0.0):
        mpm_batch_add(self._h, sim.handle, nsteps, dt, t_end)
        self.members.append(sim)

    def remove(self, sim: Simulation):
        mpm_batch_remove(self._h, sim.handle)
        self.members.remove(sim)

    def step_async(self, nsteps: int):
        mpm_batch_step_async(self._h, nsteps)

    def sync(self):
        mpm_batch_sync(self._h)

    def info(self) -> dict:
        return mpm_batch_info(self._h)

    @property
    def stream(self) -> int:
        return mpm_batch_stream(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None:
            mpm_batch_destroy(self._h)
            self._h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
