"""Python access to the FP64 CPU oracle (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The oracle is a plain serial C
implementation of the MPM step of Baioni et al. (Sec. 3, Algorithm 1); it is
compiled here with gcc and shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BC = {"wall": 0, "periodic": 1, "inflow": 2, "outflow": 3}
FIELDS = {"X": 0, "V": 1, "M": 2, "RHO": 3, "E": 4, "P": 5, "Q": 6, "ID": 7, "KEY": 8,
          "CELLSTART": 9, "GRID_M": 10, "GRID_MV": 11, "GRID_F": 12, "GRID_MV2": 13,
          "CLOCK": 14, "VBAR": 15, "GEN": 16}
ERRORS = {1: "EINVAL", 2: "ENOMEM", 4: "ESTATE", 5: "ENONFINITE", 8: "ECFL"}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {ERRORS.get(code, code)}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class _Config(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double), ("origin", C.c_double * 3),
                ("gamma", C.c_double), ("c0", C.c_double), ("c1", C.c_double), ("degree", C.c_int),
                ("bc", C.c_int * 6), ("inflow_rho", C.c_double), ("inflow_p", C.c_double),
                ("inflow_v", C.c_double * 3), ("cfl", C.c_double), ("sort_interval", C.c_int),
                ("seed", C.c_uint64), ("tile", C.c_int * 3)]


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, FP64, no contraction of a*b+c)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mpm_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-Wall", "-Wno-unused-result", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        d, i64, vp = C.c_double, C.c_int64, C.c_void_p
        L.oracle_create.argtypes = [P(_Config), P(vp)]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_destroy.restype = None
        L.oracle_add_particles.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.oracle_set_obstacle_mask.argtypes = [vp, vp, vp]
        L.oracle_cfl_dt.argtypes = [vp, P(d)]
        L.oracle_step.argtypes = [vp, i64, d, d]
        L.oracle_read.argtypes = [vp, C.c_int, vp, i64]
        L.oracle_field_size.argtypes = [vp, C.c_int]
        L.oracle_field_size.restype = i64
        L.oracle_conservation.argtypes = [vp, vp]
        L.oracle_sizes.argtypes = [vp, vp]
        L.oracle_bspline.argtypes = [C.c_int, d, vp, vp]
        L.oracle_bspline.restype = None
        L.oracle_bspline_dense.argtypes = [C.c_int, d, P(d)]
        L.oracle_bspline_dense.restype = d
        L.oracle_keys.argtypes = [P(_Config), i64, vp, C.c_int, vp]
        L.oracle_stable_sort.argtypes = [i64, vp, i64, vp, vp]
        L.oracle_reorder.argtypes = [i64, vp, vp, vp, i64, vp, vp]
        L.oracle_p2g.argtypes = [P(_Config), i64] + [vp] * 9
        L.oracle_p2g_dense.argtypes = [P(_Config), i64] + [vp] * 9
        L.oracle_p2g_fixed32.argtypes = [P(_Config), i64] + [vp] * 10
        L.oracle_obstacle_project.argtypes = [C.c_int, vp, vp, vp]
        L.oracle_obstacle_project.restype = None
        L.oracle_obstacle_profile.argtypes = [P(_Config), i64, vp, vp, vp, vp, vp]
        L.oracle_philox4x32_10.argtypes = [vp, vp, vp]
        L.oracle_philox4x32_10.restype = None
        L.oracle_riemann_exact.argtypes = [d] * 7 + [i64, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def _cfg(cfg: dict) -> _Config:
    c = _Config()
    c.dim = int(cfg["dim"])
    n = list(cfg["n"]) + [1] * (3 - len(cfg["n"]))
    c.n = (C.c_int * 3)(*[int(v) for v in n])
    c.h = float(cfg["h"])
    o = list(cfg.get("origin", [0.0, 0.0, 0.0])) + [0.0] * 3
    c.origin = (C.c_double * 3)(*[float(v) for v in o[:3]])
    c.gamma = float(cfg.get("gamma", 1.4))
    c.c0 = float(cfg.get("c0", 1.0))
    c.c1 = float(cfg.get("c1", 1.0))
    c.degree = int(cfg.get("degree", 2))
    bc = [BC[b] if isinstance(b, str) else int(b) for b in cfg["bc"]] + [0] * 6
    c.bc = (C.c_int * 6)(*bc[:6])
    c.inflow_rho = float(cfg.get("inflow_rho", 1.0))
    c.inflow_p = float(cfg.get("inflow_p", 1.0))
    iv = list(cfg.get("inflow_v", [0.0, 0.0, 0.0])) + [0.0] * 3
    c.inflow_v = (C.c_double * 3)(*[float(v) for v in iv[:3]])
    c.cfl = float(cfg.get("cfl", 0.4))
    c.sort_interval = int(cfg.get("sort_interval", 1))
    c.seed = int(cfg.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    t = list(cfg.get("tile", [0, 0, 0])) + [0, 0, 0]
    c.tile = (C.c_int * 3)(*[int(v) for v in t[:3]])
    return c


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(code: int, what: str):
    if code != 0:
        raise OracleError(code, what)


class OracleSim:
    """The FP64 oracle simulation, same life cycle as the product's handle."""

    def __init__(self, cfg: dict):
        self._L = lib()
        self.cfg = dict(cfg)
        self.dim = int(cfg["dim"])
        self._c = _cfg(cfg)
        h = C.c_void_p()
        _check(self._L.oracle_create(C.byref(self._c), C.byref(h)), "create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.oracle_destroy(self._h)
            self._h = None

    __del__ = close

    def add_particles(self, x, v, mass, rho, e):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        n = int(mass.shape[0])
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (mass, rho, e)]
        _check(self._L.oracle_add_particles(self._h, n, _ptr(x), _ptr(v), *[_ptr(a) for a in arrs]),
               "add_particles")

    def set_obstacle_mask(self, mask, normals):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        normals = np.ascontiguousarray(normals, dtype=np.float64)
        _check(self._L.oracle_set_obstacle_mask(self._h, _ptr(mask), _ptr(normals)), "set_obstacle_mask")

    def cfl_dt(self) -> float:
        out = C.c_double()
        _check(self._L.oracle_cfl_dt(self._h, C.byref(out)), "cfl_dt")
        return out.value

    def step(self, nsteps: int, dt: float = 0.0, t_end: float = 0.0):
        _check(self._L.oracle_step(self._h, int(nsteps), float(dt), float(t_end)), "step")

    def read(self, field: str) -> np.ndarray:
        f = FIELDS[field]
        n = int(self._L.oracle_field_size(self._h, f))
        out = np.empty(n, dtype=np.float64)
        _check(self._L.oracle_read(self._h, f, _ptr(out), n), "read")
        if field in ("X", "V", "VBAR"):
            out = out.reshape(self.dim, -1)
        elif field in ("GRID_MV", "GRID_F", "GRID_MV2"):
            out = out.reshape(self.dim, -1)
        return out

    def conservation(self) -> np.ndarray:
        out = np.empty(5, dtype=np.float64)
        _check(self._L.oracle_conservation(self._h, _ptr(out)), "conservation")
        return out

    def sizes(self):
        out = np.empty(4, dtype=np.int64)
        _check(self._L.oracle_sizes(self._h, _ptr(out)), "sizes")
        return {"particles": int(out[0]), "nodes": int(out[1]), "keys": int(out[2]), "steps": int(out[3])}


# ---------------------------------------------------------------- unit pieces

def bspline(degree: int, fx: float):
    w = np.zeros(3)
    dw = np.zeros(3)
    lib().oracle_bspline(int(degree), float(fx), _ptr(w), _ptr(dw))
    return w, dw


def bspline_dense(degree: int, r: float):
    dn = C.c_double()
    v = lib().oracle_bspline_dense(int(degree), float(r), C.byref(dn))
    return v, dn.value


def keys(cfg: dict, x: np.ndarray, prec32: bool = False) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[1]
    out = np.empty(n, dtype=np.uint32)
    c = _cfg(cfg)
    _check(lib().oracle_keys(C.byref(c), n, _ptr(x), int(bool(prec32)), _ptr(out)), "keys")
    return out


def stable_sort(k: np.ndarray, nkeys: int):
    k = np.ascontiguousarray(k, dtype=np.uint32)
    perm = np.empty(k.shape[0], dtype=np.int64)
    start = np.empty(nkeys + 1, dtype=np.int64)
    _check(lib().oracle_stable_sort(k.shape[0], _ptr(k), int(nkeys), _ptr(perm), _ptr(start)), "stable_sort")
    return perm, start


def reorder(k: np.ndarray, recycled: np.ndarray, ids: np.ndarray, nkeys: int):
    """The per-step re-order (Sec. 3 step xii) of particles in their current
    order: perm[j] = current index placed at j, start = first position of
    each key.  Particles with recycled != 0 (re-created at the inflow in the
    step) follow the others of their key, by id."""
    k = np.ascontiguousarray(k, dtype=np.uint32)
    r = np.ascontiguousarray(recycled, dtype=np.uint8)
    i = np.ascontiguousarray(ids, dtype=np.int64)
    perm = np.empty(k.shape[0], dtype=np.int64)
    start = np.empty(nkeys + 1, dtype=np.int64)
    _check(lib().oracle_reorder(k.shape[0], _ptr(k), _ptr(r), _ptr(i), int(nkeys), _ptr(perm), _ptr(start)),
           "reorder")
    return perm, start


def _grid_sizes(cfg: dict):
    s = OracleSim(cfg)
    z = s.sizes()
    s.close()
    return z["nodes"], z["keys"]


def obstacle_profile(cfg: dict, loops):
    """Node mask, normals (2, nodes) and signed distance of a 2D obstacle given
    as closed loops of boundary points, each a (2, k) array (Eq. sdf)."""
    loops = [np.asarray(l, dtype=np.float64) for l in loops]
    lens = np.array([l.shape[1] for l in loops], dtype=np.int64)
    pts = np.ascontiguousarray(np.concatenate(loops, axis=1))
    nn, _ = _grid_sizes(cfg)
    mask = np.empty(nn, dtype=np.uint8)
    nrm = np.empty(2 * nn)
    sd = np.empty(nn)
    _check(lib().oracle_obstacle_profile(C.byref(_cfg(cfg)), len(loops), _ptr(lens), _ptr(pts), _ptr(mask),
                                         _ptr(nrm), _ptr(sd)), "obstacle_profile")
    return mask, nrm.reshape(2, nn), sd


def p2g(cfg: dict, x, v, mass, rho, e, q=None, dense: bool = False):
    d = int(cfg["dim"])
    nn, _ = _grid_sizes(cfg)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (mass, rho, e)]
    qa = np.ascontiguousarray(q, dtype=np.float64) if q is not None else np.zeros_like(arrs[0])
    gm = np.empty(nn)
    gmv = np.empty(d * nn)
    gf = np.empty(d * nn)
    c = _cfg(cfg)
    fn = lib().oracle_p2g_dense if dense else lib().oracle_p2g
    _check(fn(C.byref(c), arrs[0].shape[0], _ptr(x), _ptr(v), *[_ptr(a) for a in arrs], _ptr(qa),
              _ptr(gm), _ptr(gmv), _ptr(gf)), "p2g")
    return gm, gmv.reshape(d, nn), gf.reshape(d, nn)


def p2g_fixed32(cfg: dict, x, v, mass, rho, e, q=None, unit=(1.0, 1.0, 1.0)):
    d = int(cfg["dim"])
    nn, _ = _grid_sizes(cfg)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    x, v, mass, rho, e = f32(x), f32(v), f32(mass), f32(rho), f32(e)
    qa = f32(q) if q is not None else np.zeros_like(mass)
    u = np.ascontiguousarray(unit, dtype=np.float64)
    gm = np.empty(nn, dtype=np.int64)
    gmv = np.empty(d * nn, dtype=np.int64)
    gf = np.empty(d * nn, dtype=np.int64)
    c = _cfg(cfg)
    _check(lib().oracle_p2g_fixed32(C.byref(c), mass.shape[0], _ptr(x), _ptr(v), _ptr(mass), _ptr(rho),
                                    _ptr(e), _ptr(qa), _ptr(u), _ptr(gm), _ptr(gmv), _ptr(gf)), "p2g_fixed32")
    return gm, gmv.reshape(d, nn), gf.reshape(d, nn)


def obstacle_project(x, n):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    out = np.empty_like(x)
    lib().oracle_obstacle_project(x.shape[0], _ptr(x), _ptr(n), _ptr(out))
    return out


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def riemann_exact(gamma, left, right, s):
    s = np.ascontiguousarray(s, dtype=np.float64)
    rho, u, p = np.empty_like(s), np.empty_like(s), np.empty_like(s)
    star = np.empty(2)
    _check(lib().oracle_riemann_exact(float(gamma), *map(float, left), *map(float, right), s.shape[0],
                                      _ptr(s), _ptr(rho), _ptr(u), _ptr(p), _ptr(star)), "riemann_exact")
    return rho, u, p, star
