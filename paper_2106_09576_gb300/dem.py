"""Thin ctypes binding of libdem_gb300.so (include/dem.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  PyTorch provides the
device workspace (one uint8 tensor) and the stream.  There is no CPU path: if the
library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DEM_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_CAPACITY", 4: "ERR_NONFINITE",
                5: "ERR_OVERLAP", 6: "ERR_TIMEOUT", 7: "ERR_STATE"}
PRECISION = {"fp64": 0, "mixed": 1}
PAIR_EVAL = {"once": 0, "both": 1}
EXPORTED = ["dem_workspace_bytes", "dem_create", "dem_set_walls", "dem_step", "dem_step_profiled", "dem_sync",
            "dem_get_state",
            "dem_set_state", "dem_get_forces", "dem_get_pairs", "dem_get_history", "dem_set_history",
            "dem_get_stats", "dem_status_string", "dem_destroy", "dem_find_pairs_static", "dem_set_instances",
            "dem_pipe_rates"]
MAX_INSTANCE_WALLS = 4


class DemError(RuntimeError):
    def __init__(self, call, code, msg):
        super().__init__(f"{call} failed: {STATUS_NAMES.get(code, code)} ({msg})")
        self.code = code


class Material(C.Structure):
    _fields_ = [("young", C.c_double), ("poisson", C.c_double), ("restitution", C.c_double),
                ("mu_slide", C.c_double), ("mu_roll", C.c_double)]


class Config(C.Structure):
    _fields_ = [("n", C.c_int64), ("density", C.c_double), ("radius_max", C.c_double),
                ("particle", Material), ("wall", Material), ("gravity", C.c_double * 3),
                ("dt", C.c_double), ("neighbor_factor", C.c_double), ("skin", C.c_double),
                ("rebuild_every", C.c_int32), ("precision", C.c_int32), ("rolling_model", C.c_int32),
                ("n_instances", C.c_int32), ("domain_lo", C.c_double * 3), ("domain_hi", C.c_double * 3),
                ("z_sink", C.c_double), ("max_overlap_ratio", C.c_double), ("step_block", C.c_int32),
                ("contact_model", C.c_int32), ("integrator", C.c_int32), ("pair_eval", C.c_int32),
                ("linear_velocity", C.c_double)]


class Wall(C.Structure):
    _fields_ = [("kind", C.c_int32), ("translates", C.c_int32), ("point", C.c_double * 3),
                ("normal", C.c_double * 3), ("radius", C.c_double), ("inner_radius", C.c_double),
                ("omega", C.c_double), ("rot_origin", C.c_double * 3), ("rot_axis", C.c_double * 3),
                ("velocity", C.c_double * 3), ("t_on", C.c_double), ("t_off", C.c_double)]


class Instance(C.Structure):
    _fields_ = [("first", C.c_int64), ("particle", Material), ("wall", Material), ("n_walls", C.c_int32),
                ("reserved0", C.c_int32), ("walls", Wall * MAX_INSTANCE_WALLS)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("rebuilds", C.c_int64), ("n_pairs", C.c_int64),
                ("n_touch", C.c_int64), ("n_wall_touch", C.c_int64), ("n_active", C.c_int64),
                ("time", C.c_double), ("max_overlap_ratio", C.c_double), ("status_bits", C.c_uint32),
                ("max_neighbors_seen", C.c_int32), ("required_workspace", C.c_size_t),
                ("inner_builds", C.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads libdem_gb300.so; builds it first if it is absent (nvcc required)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is missing: run paper_2106_09576_gb300.build.build()")
        _build.build()
    lib = C.CDLL(_build.LIB)
    P = C.c_void_p
    S = C.c_int32
    sig = {
        "dem_workspace_bytes": [C.POINTER(Config), C.POINTER(C.c_size_t)],
        "dem_create": [C.POINTER(Config), P, P, P, P, P, C.c_size_t, P, C.POINTER(P)],
        "dem_set_walls": [P, C.POINTER(Wall), C.c_int32],
        "dem_step": [P, C.c_int64],
        "dem_sync": [P],
        "dem_step_profiled": [P, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                              C.POINTER(C.c_int64)],
        "dem_get_state": [P, P, P, P, P],
        "dem_set_state": [P, P, P, P, P],
        "dem_get_forces": [P, P, P],
        "dem_get_pairs": [P, P, C.c_int64, C.POINTER(C.c_int64)],
        "dem_get_history": [P, P, P, C.c_int64, C.POINTER(C.c_int64), P],
        "dem_set_history": [P, C.c_int64, P, P, P],
        "dem_get_stats": [P, C.POINTER(Stats)],
        "dem_set_instances": [P, C.POINTER(Instance), C.c_int32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = S
    lib.dem_status_string.argtypes = [S]
    lib.dem_status_string.restype = C.c_char_p
    lib.dem_destroy.argtypes = [P]
    lib.dem_destroy.restype = None
    _lib = lib
    return lib


def _check(lib, call, code):
    if code != DEM_OK:
        raise DemError(call, code, lib.dem_status_string(code).decode())


def _ptr(a):
    """Pointer of a NumPy array or a torch tensor (host or device), or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _material(d) -> Material:
    return Material(d["young"], d["poisson"], d["restitution"], d["mu_slide"], d["mu_roll"])


def make_config(cfg: dict, n: int, radius_max: float, precision=None) -> Config:
    c = Config()
    c.n = n
    c.density = cfg["density"]
    c.radius_max = float(radius_max)
    c.particle = _material(cfg["particle"])
    c.wall = _material(cfg.get("wall", cfg["particle"]))
    c.gravity[:] = list(cfg.get("gravity", (0.0, 0.0, -9.81)))
    c.dt = cfg["dt"]
    c.neighbor_factor = cfg.get("neighbor_factor", 1.3)
    c.skin = cfg.get("skin", 0.0)
    c.rebuild_every = cfg.get("rebuild_every", 0)
    prec = precision if precision is not None else cfg.get("precision", "fp64")
    c.precision = PRECISION[prec] if isinstance(prec, str) else int(prec)
    c.rolling_model = cfg.get("rolling_model", 1)
    c.domain_lo[:] = list(cfg["domain_lo"])
    c.domain_hi[:] = list(cfg["domain_hi"])
    c.z_sink = cfg.get("z_sink", -1e300)
    c.max_overlap_ratio = cfg.get("max_overlap_ratio", 0.0)
    c.n_instances = int(cfg.get("n_instances", len(cfg.get("instances", ()))))
    c.step_block = int(cfg.get("step_block", 0))
    c.contact_model = int(cfg.get("contact_model", 0))
    c.integrator = int(cfg.get("integrator", 0))
    c.linear_velocity = float(cfg.get("linear_velocity", 1.0))
    pe = cfg.get("pair_eval", "once")
    c.pair_eval = PAIR_EVAL[pe] if isinstance(pe, str) else int(pe)
    return c


def _fill_wall(W, w):
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


def make_instances(instances):
    """dem_instance array from dicts {first, particle, wall, walls}."""
    arr = (Instance * len(instances))()
    for k, d in enumerate(instances):
        I = arr[k]
        I.first = int(d["first"])
        I.particle = _material(d["particle"])
        I.wall = _material(d.get("wall", d["particle"]))
        I.n_walls = len(d["walls"])
        if I.n_walls > MAX_INSTANCE_WALLS:
            raise ValueError(f"instance {k}: more than {MAX_INSTANCE_WALLS} walls")
        for w, wd in enumerate(d["walls"]):
            _fill_wall(I.walls[w], wd)
    return arr


def make_walls(walls):
    arr = (Wall * max(1, len(walls)))()
    for k, w in enumerate(walls):
        _fill_wall(arr[k], w)
    return arr, len(walls)


def find_pairs_static(x, cutoff: float, domain_lo, domain_hi, active=None, out=None, stream=None):
    """dem_find_pairs_static: contact search without any device allocation by the library.

    For callers that cannot allocate device memory; `x` ([n, 3] float64, contiguous) and
    `active` ([n] uint8, optional) are CUDA tensors on one device, which is made current
    for the call.  With `out` (a contiguous CUDA int32 tensor [capacity, 2]) the call
    writes the first min(count, capacity) pairs into it, allocates nothing, and returns
    the total count.  Without it, a tensor of exactly count rows is allocated here by
    torch on the caller's behalf (one counting call, one writing call) and returned."""
    import torch

    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.dim() == 2
            and x.shape[1] == 3 and x.is_contiguous()):
        raise ValueError("x must be a contiguous CUDA float64 tensor of shape [n, 3]")
    n = int(x.shape[0])
    if active is not None and not (isinstance(active, torch.Tensor) and active.device == x.device
                                   and active.dtype == torch.uint8 and active.shape == (n,)
                                   and active.is_contiguous()):
        raise ValueError("active must be a contiguous uint8 tensor of shape [n] on x's device")
    if out is not None and not (isinstance(out, torch.Tensor) and out.device == x.device and out.dtype == torch.int32
                                and out.dim() == 2 and out.shape[1] == 2 and out.is_contiguous()):
        raise ValueError("out must be a contiguous int32 tensor of shape [capacity, 2] on x's device")
    lib = load_library()
    f = lib.dem_find_pairs_static
    if f.argtypes is None:
        f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.POINTER(C.c_double),
                      C.POINTER(C.c_double), C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]
        f.restype = C.c_int32
    lo = (C.c_double * 3)(*[float(v) for v in domain_lo])
    hi = (C.c_double * 3)(*[float(v) for v in domain_hi])
    with torch.cuda.device(x.device):
        st = stream if stream is not None else torch.cuda.current_stream(x.device)
        sp = C.c_void_p(st.cuda_stream)
        cnt = C.c_int64(0)
        a = None if active is None else C.c_void_p(active.data_ptr())
        xp = C.c_void_p(x.data_ptr())
        if out is not None:
            cap = int(out.shape[0])
            _check(lib, "dem_find_pairs_static", f(xp, a, n, float(cutoff), lo, hi,
                                                    C.c_void_p(out.data_ptr()) if cap else None, cap,
                                                    C.byref(cnt), sp))
            return int(cnt.value)
        _check(lib, "dem_find_pairs_static", f(xp, a, n, float(cutoff), lo, hi, None, 0, C.byref(cnt), sp))
        res = torch.empty((max(cnt.value, 1), 2), dtype=torch.int32, device=x.device)
        if cnt.value:
            _check(lib, "dem_find_pairs_static", f(xp, a, n, float(cutoff), lo, hi, C.c_void_p(res.data_ptr()),
                                                    cnt.value, C.byref(cnt), sp))
        return res[: cnt.value]


def pipe_rates(device=None):
    """dem_pipe_rates on `device` (default: the current one): measured thread-level
    instructions per second of FP64 FMA, FP64 add, FP32 FMA and FP32 -> FP64 conversion."""
    import torch

    lib = load_library()
    f = lib.dem_pipe_rates
    f.argtypes = [C.c_void_p, C.c_void_p]
    f.restype = C.c_int32
    out = (C.c_double * 4)()
    dev = torch.device("cuda") if device is None else torch.device(device)
    with torch.cuda.device(dev):
        _check(lib, "dem_pipe_rates", f(out, C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))
    return {"dfma": out[0], "dadd": out[1], "ffma": out[2], "f2d": out[3]}


def history_arrays(pairs, dt_pair, dt_wall, n: int, n_walls: int):
    """Host arrays for dem_set_history, checked against the shapes the call reads: pairs
    [k][2] int32 of particle indices, dt_pair [k][3] and dt_wall [n][n_walls][3] float64."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    dt_pair = np.ascontiguousarray(dt_pair, dtype=np.float64)
    if dt_pair.size != 3 * len(pairs):
        raise ValueError(f"dt_pair holds {dt_pair.size} values for {len(pairs)} pairs (3 per pair)")
    dt_pair = dt_pair.reshape(-1, 3)
    if len(pairs) and (pairs.min() < 0 or pairs.max() >= n):
        raise ValueError(f"pair indices outside [0, {n})")
    dtw = None
    if dt_wall is not None:
        dtw = np.ascontiguousarray(dt_wall, dtype=np.float64)
        if dtw.shape != (n, n_walls, 3):
            raise ValueError(f"dt_wall has shape {dtw.shape}, expected {(n, n_walls, 3)}")
    return pairs, dt_pair, dtw


def _host(a, dtype, shape):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a.reshape(shape)


class DEM:
    """One simulation context.  Inputs may be NumPy arrays or torch tensors (CPU or CUDA)."""

    def __init__(self, cfg: dict, x, v, w, radius, walls=(), precision=None, device=None, stream=None):
        import torch

        self.lib = load_library()
        n = int(radius.shape[0])
        self.n = n
        if hasattr(radius, "detach"):
            rmax = float(radius.detach().max().cpu())
        else:
            rmax = float(np.max(radius))
        self._cfg = make_config(cfg, n, rmax, precision)
        self.device = torch.device(device if device is not None else "cuda")
        size = C.c_size_t(0)
        _check(self.lib, "dem_workspace_bytes", self.lib.dem_workspace_bytes(C.byref(self._cfg), C.byref(size)))
        self.workspace = torch.empty(int(size.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        keep = [self._prep(a, np.float64, (n, 3)) for a in (x, v, w)]
        r = self._prep(radius, np.float32, (n,))
        h = C.c_void_p()
        _check(self.lib, "dem_create", self.lib.dem_create(
            C.byref(self._cfg), _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]), _ptr(r),
            C.c_void_p(self.workspace.data_ptr()), size.value, C.c_void_p(self.stream.cuda_stream),
            C.byref(h)))
        self.h = h
        self.n_walls = 0
        if walls:
            self.set_walls(walls)
        if cfg.get("instances"):
            self.set_instances(cfg["instances"])

    @staticmethod
    def _prep(a, dtype, shape):
        if hasattr(a, "data_ptr"):
            import torch
            tdt = {np.float64: torch.float64, np.float32: torch.float32, np.uint8: torch.uint8}[dtype]
            return a.detach().to(tdt).contiguous().reshape(shape)
        return _host(a, dtype, shape)

    def close(self):
        if getattr(self, "h", None):
            self.lib.dem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_walls(self, walls):
        arr, k = make_walls(list(walls))
        _check(self.lib, "dem_set_walls", self.lib.dem_set_walls(self.h, arr, k))
        self.n_walls = k

    def set_instances(self, instances):
        """Batch contexts: per-instance particle ranges, materials and walls (dicts with keys
        first, particle, wall, walls)."""
        arr = make_instances(list(instances))
        _check(self.lib, "dem_set_instances", self.lib.dem_set_instances(self.h, arr, len(instances)))

    def step(self, n_steps: int = 1):
        _check(self.lib, "dem_step", self.lib.dem_step(self.h, int(n_steps)))

    def step_profiled(self, n_steps: int):
        """Same steps as step(), launched one by one with CUDA events around the step
        kernel and the contact searches; returns the device milliseconds and counts."""
        ks, ss, is_ = C.c_double(0), C.c_double(0), C.c_double(0)
        nk, ns, ni = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        _check(self.lib, "dem_step_profiled", self.lib.dem_step_profiled(
            self.h, int(n_steps), C.byref(ks), C.byref(ss), C.byref(nk), C.byref(ns), C.byref(is_), C.byref(ni)))
        return dict(step_kernel_ms=ks.value, search_ms=ss.value, step_launches=nk.value, searches=ns.value,
                    inner_ms=is_.value, inner_builds=ni.value)

    def sync(self):
        _check(self.lib, "dem_sync", self.lib.dem_sync(self.h))

    def state(self, out=None):
        """Returns (x, v, w, active) as NumPy arrays, or fills the given torch tensors."""
        if out is None:
            x = np.empty((self.n, 3)); v = np.empty((self.n, 3)); w = np.empty((self.n, 3))
            a = np.empty(self.n, dtype=np.uint8)
        else:
            x, v, w, a = out
        _check(self.lib, "dem_get_state", self.lib.dem_get_state(self.h, _ptr(x), _ptr(v), _ptr(w), _ptr(a)))
        if out is None:
            return x, v, w, a.astype(bool)
        return out

    def set_state(self, x=None, v=None, w=None, active=None):
        n = self.n
        keep = [None if a is None else self._prep(a, np.float64, (n, 3)) for a in (x, v, w)]
        act = None if active is None else self._prep(active, np.uint8, (n,))
        _check(self.lib, "dem_set_state",
               self.lib.dem_set_state(self.h, _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]), _ptr(act)))

    def forces(self):
        F = np.empty((self.n, 3)); M = np.empty((self.n, 3))
        _check(self.lib, "dem_get_forces", self.lib.dem_get_forces(self.h, _ptr(F), _ptr(M)))
        return F, M

    def pairs(self) -> np.ndarray:
        cnt = C.c_int64(0)
        _check(self.lib, "dem_get_pairs", self.lib.dem_get_pairs(self.h, None, 0, C.byref(cnt)))
        out = np.empty((max(cnt.value, 1), 2), dtype=np.int32)
        _check(self.lib, "dem_get_pairs", self.lib.dem_get_pairs(self.h, _ptr(out), cnt.value, C.byref(cnt)))
        out = out[: cnt.value]
        return out[np.lexsort((out[:, 1], out[:, 0]))]

    def history(self):
        cnt = C.c_int64(0)
        _check(self.lib, "dem_get_history",
               self.lib.dem_get_history(self.h, None, None, 0, C.byref(cnt), None))
        pairs = np.empty((max(cnt.value, 1), 2), dtype=np.int32)
        vals = np.empty((max(cnt.value, 1), 3))
        dtw = np.zeros((self.n, max(self.n_walls, 1), 3))
        _check(self.lib, "dem_get_history", self.lib.dem_get_history(
            self.h, _ptr(pairs), _ptr(vals), cnt.value, C.byref(cnt), _ptr(dtw) if self.n_walls else None))
        pairs, vals = pairs[: cnt.value], vals[: cnt.value]
        o = np.lexsort((pairs[:, 1], pairs[:, 0]))
        return pairs[o], vals[o], dtw[:, : self.n_walls]

    def set_history(self, pairs, dt_pair, dt_wall=None):
        pairs, dt_pair, dtw = history_arrays(pairs, dt_pair, dt_wall, self.n, self.n_walls)
        _check(self.lib, "dem_set_history",
               self.lib.dem_set_history(self.h, len(pairs), _ptr(pairs), _ptr(dt_pair), _ptr(dtw)))

    def stats(self) -> dict:
        s = Stats()
        _check(self.lib, "dem_get_stats", self.lib.dem_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}
