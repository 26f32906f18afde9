"""CPU oracle of the soft-sphere DEM time step (Golshan et al., Lethe-DEM, arXiv 2106.09576).

TEST INFRASTRUCTURE ONLY.  This package is the plain FP64 C restatement of the method
(``dem_oracle.c``) and its ctypes loader.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA library and never imports it.

Inputs are NumPy arrays: positions, velocities and angular velocities ``[n, 3]`` FP64,
radii ``[n]`` FP32.  Configuration and walls are plain dicts (the keys of the workload
generators in ``workloads/``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_dem.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no floating-point contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    hdr = os.path.join(_HERE, "dem_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Material(C.Structure):
    _fields_ = [("young", C.c_double), ("poisson", C.c_double), ("restitution", C.c_double),
                ("mu_slide", C.c_double), ("mu_roll", C.c_double)]


class Config(C.Structure):
    _fields_ = [("n", C.c_int64), ("density", C.c_double), ("particle", Material),
                ("wall", Material), ("gravity", C.c_double * 3), ("dt", C.c_double),
                ("neighbor_factor", C.c_double), ("skin", C.c_double),
                ("rebuild_every", C.c_int32), ("rolling_model", C.c_int32),
                ("contact_model", C.c_int32), ("integrator", C.c_int32), ("linear_velocity", C.c_double),
                ("domain_lo", C.c_double * 3), ("domain_hi", C.c_double * 3),
                ("z_sink", C.c_double)]


class Wall(C.Structure):
    _fields_ = [("kind", C.c_int32), ("translates", C.c_int32), ("point", C.c_double * 3), ("normal", C.c_double * 3),
                ("radius", C.c_double), ("inner_radius", C.c_double), ("omega", C.c_double),
                ("rot_origin", C.c_double * 3), ("rot_axis", C.c_double * 3),
                ("velocity", C.c_double * 3), ("t_on", C.c_double), ("t_off", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("rebuilds", C.c_int64), ("n_pairs", C.c_int64),
                ("n_touch", C.c_int64), ("n_wall_touch", C.c_int64), ("n_active", C.c_int64),
                ("time", C.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = _bind(C.CDLL(_LIB_PATH))
    return _lib


class swap_library:
    """Context manager: use another build of the oracle (e.g. a copy with a planted
    mistake, compiled by the test suite) for the duration of a block."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = _bind(C.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a variant of the oracle source with the same flags (test use only)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-I", _HERE, "-o", out_path, src, "-lm"])
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _bind(lib):
    P = C.c_void_p
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [C.POINTER(Config), P, P, P, P]
    lib.orc_destroy.argtypes = [P]
    lib.orc_set_walls.argtypes = [P, C.POINTER(Wall), C.c_int32]
    lib.orc_step.argtypes = [P, C.c_int64]
    lib.orc_get_state.argtypes = [P, P, P, P, P]
    lib.orc_set_state.argtypes = [P, P, P, P, P]
    lib.orc_get_forces.argtypes = [P, P, P]
    lib.orc_get_force_scales.argtypes = [P, P, P]
    lib.orc_get_pairs.restype = C.c_int64
    lib.orc_get_pairs.argtypes = [P, P, C.c_int64]
    lib.orc_get_history.restype = C.c_int64
    lib.orc_get_history.argtypes = [P, P, P, C.c_int64, P]
    lib.orc_set_history.argtypes = [P, C.c_int64, P, P, P]
    lib.orc_get_stats.argtypes = [P, C.POINTER(Stats)]
    lib.orc_brute_pairs.restype = C.c_int64
    lib.orc_brute_pairs.argtypes = [C.c_int64, P, P, C.c_double, P, C.c_int64]
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _material(d) -> Material:
    return Material(d["young"], d["poisson"], d["restitution"], d["mu_slide"], d["mu_roll"])


def make_config(cfg: dict, n: int) -> Config:
    c = Config()
    c.n = n
    c.density = cfg["density"]
    c.particle = _material(cfg["particle"])
    c.wall = _material(cfg.get("wall", cfg["particle"]))
    c.gravity[:] = list(cfg.get("gravity", (0.0, 0.0, -9.81)))
    c.dt = cfg["dt"]
    c.neighbor_factor = cfg.get("neighbor_factor", 1.3)
    c.skin = cfg.get("skin", 0.0)
    c.rebuild_every = cfg.get("rebuild_every", 0)
    c.rolling_model = cfg.get("rolling_model", 1)
    c.contact_model = cfg.get("contact_model", 0)
    c.integrator = cfg.get("integrator", 0)
    c.linear_velocity = cfg.get("linear_velocity", 1.0)
    c.domain_lo[:] = list(cfg["domain_lo"])
    c.domain_hi[:] = list(cfg["domain_hi"])
    c.z_sink = cfg.get("z_sink", -1e300)
    return c


def make_walls(walls) -> tuple:
    arr = (Wall * max(1, len(walls)))()
    for k, w in enumerate(walls):
        W = arr[k]
        W.kind = w["kind"]
        W.translates = int(w.get("translates", 0))
        W.point[:] = list(w["point"])
        W.normal[:] = list(w["normal"])
        W.radius = w.get("radius", 0.0)
        W.inner_radius = w.get("inner_radius", 0.0)
        W.omega = w.get("omega", 0.0)
        W.rot_origin[:] = list(w.get("rot_origin", (0.0, 0.0, 0.0)))
        W.rot_axis[:] = list(w.get("rot_axis", (0.0, 0.0, 1.0)))
        W.velocity[:] = list(w.get("velocity", (0.0, 0.0, 0.0)))
        W.t_on = w.get("t_on", -1e300)
        W.t_off = w.get("t_off", 1e300)
    return arr, len(walls)


class OracleSim:
    """One oracle simulation (a thin ctypes handle; all arithmetic is in dem_oracle.c)."""

    def __init__(self, cfg: dict, x, v, w, radius, walls=()):
        self.lib = _load()
        self.n = int(len(radius))
        self.x0 = np.ascontiguousarray(x, dtype=np.float64).reshape(self.n, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(self.n, 3)
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(self.n, 3)
        r = np.ascontiguousarray(radius, dtype=np.float32)
        self._cfg = make_config(cfg, self.n)
        self.h = self.lib.orc_create(C.byref(self._cfg), _ptr(self.x0), _ptr(v), _ptr(w), _ptr(r))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        self.n_walls = 0
        if walls:
            self.set_walls(walls)

    def close(self):
        if self.h:
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_walls(self, walls):
        arr, k = make_walls(list(walls))
        if self.lib.orc_set_walls(self.h, arr, k) != 0:
            raise ValueError("oracle rejected the walls")
        self.n_walls = k

    def step(self, n_steps: int = 1):
        if self.lib.orc_step(self.h, int(n_steps)) != 0:
            raise RuntimeError("orc_step failed")

    def state(self):
        x = np.empty((self.n, 3)); v = np.empty((self.n, 3)); w = np.empty((self.n, 3))
        a = np.empty(self.n, dtype=np.uint8)
        self.lib.orc_get_state(self.h, _ptr(x), _ptr(v), _ptr(w), _ptr(a))
        return x, v, w, a.astype(bool)

    def set_state(self, x=None, v=None, w=None, active=None):
        def c(a, dt):
            return None if a is None else np.ascontiguousarray(a, dtype=dt)
        x, v, w = c(x, np.float64), c(v, np.float64), c(w, np.float64)
        active = c(active, np.uint8)
        self.lib.orc_set_state(self.h, _ptr(x), _ptr(v), _ptr(w), _ptr(active))

    def forces(self):
        F = np.empty((self.n, 3)); M = np.empty((self.n, 3))
        self.lib.orc_get_forces(self.h, _ptr(F), _ptr(M))
        return F, M

    def force_scales(self):
        """Per particle: sum of |contact force| and of |contact torque| (error scales)."""
        Fa = np.empty(self.n); Ma = np.empty(self.n)
        self.lib.orc_get_force_scales(self.h, _ptr(Fa), _ptr(Ma))
        return Fa, Ma

    def pairs(self) -> np.ndarray:
        cnt = self.lib.orc_get_pairs(self.h, None, 0)
        out = np.empty((max(cnt, 1), 2), dtype=np.int32)
        self.lib.orc_get_pairs(self.h, _ptr(out), cnt)
        return out[:cnt]

    def history(self):
        cnt = self.lib.orc_get_history(self.h, None, None, 0, None)
        pairs = np.empty((max(cnt, 1), 2), dtype=np.int32)
        dtp = np.empty((max(cnt, 1), 3))
        dtw = np.empty((self.n, max(self.n_walls, 1), 3))
        self.lib.orc_get_history(self.h, _ptr(pairs), _ptr(dtp), cnt, _ptr(dtw))
        return pairs[:cnt], dtp[:cnt], dtw[:, : self.n_walls]

    def set_history(self, pairs, dt_pair, dt_wall=None):
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        dt_pair = np.ascontiguousarray(dt_pair, dtype=np.float64).reshape(-1, 3)
        dtw = None if dt_wall is None else np.ascontiguousarray(dt_wall, dtype=np.float64)
        if self.lib.orc_set_history(self.h, len(pairs), _ptr(pairs), _ptr(dt_pair), _ptr(dtw)) != 0:
            raise ValueError("oracle rejected the history")

    def stats(self) -> dict:
        s = Stats()
        self.lib.orc_get_stats(self.h, C.byref(s))
        return {k: getattr(s, k) for k, _ in Stats._fields_}


def brute_pairs(x, rc: float, active=None) -> np.ndarray:
    """All pairs i < j with |x_j - x_i|^2 < rc^2 by the O(n^2) loop in dem_oracle.c."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    n = len(x)
    a = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
    cnt = lib.orc_brute_pairs(n, _ptr(x), _ptr(a), float(rc), None, 0)
    out = np.empty((max(cnt, 1), 2), dtype=np.int32)
    lib.orc_brute_pairs(n, _ptr(x), _ptr(a), float(rc), _ptr(out), cnt)
    return out[:cnt]
