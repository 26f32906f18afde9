"""Binding and driver of the learned surrogate (include/surrogate.h).

A message-passing network on the radius-1.2 d contact graph of a rotating drum predicts
each particle's velocity and spin increments over k = 10 DEM steps.  Every computation --
graph, features, forward and backward passes, loss, optimiser, rollout -- runs in the
library's CUDA kernels; this module only marshals arguments and sequences the calls.
Training data come from DEM trajectories of the drum computed by the library itself; the
rollout falls back to plain DEM steps when the surrogate's state shows too much overlap or
a kinetic-energy jump.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import dem as _dem

K_STEPS = 10
SURR_FUNCS = ["surr_params", "surr_workspace_bytes", "surr_build_csr", "surr_params_to_bf16", "surr_forward",
              "surr_backward", "surr_mse", "surr_adam", "surr_gemm_bf16", "surr_features", "surr_targets",
              "surr_apply"]


class Layout(C.Structure):
    _fields_ = [("W", C.c_int64 * 6), ("b", C.c_int64 * 6), ("total", C.c_int64)]


_bound = None


def lib():
    global _bound
    if _bound is not None:
        return _bound
    L = _dem.load_library()
    P, I64, I32, F, D = C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_double
    sig = {
        "surr_params": [C.POINTER(Layout)],
        "surr_workspace_bytes": [I64, I64, C.POINTER(C.c_size_t)],
        "surr_build_csr": [P, I64, I64, P, P, P, P],
        "surr_params_to_bf16": [P, P, I64, P],
        "surr_forward": [P, P, P, P, P, P, I64, I64, P, P, P],
        "surr_backward": [P, P, P, P, I64, I64, P, P, P],
        "surr_mse": [P, P, P, I64, P, P, P],
        "surr_adam": [P, P, P, P, P, I64, F, F, F, F, I64, P],
        "surr_gemm_bf16": [P, P, P, I64, I64, I64, P],
        "surr_features": [P, P, P, P, I64, P, P, I64, P, P, P, P, P],
        "surr_targets": [P, P, P, P, P, I64, P, P, P, P],
        "surr_apply": [P, P, P, P, I64, P, P, P, D, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    _bound = L
    return L


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _ok(name, code):
    if code != 0:
        raise RuntimeError(f"{name} failed with code {code}")


def _stream(torch, dev):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def param_layout():
    lay = Layout()
    _ok("surr_params", lib().surr_params(C.byref(lay)))
    return [(lay.W[l], lay.b[l]) for l in range(6)], lay.total


class Graph:
    """Receiver-sorted CSR of the radius graph of positions x (CUDA [n][3] float64)."""

    def __init__(self, x, cutoff, lo, hi):
        import torch
        pairs = _dem.find_pairs_static(x, cutoff, lo, hi)
        n = int(x.shape[0])
        self.n = n
        self.n_edges = 2 * int(pairs.shape[0])
        dev = x.device
        self.row_ptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
        self.col = torch.empty(max(self.n_edges, 1), dtype=torch.int32, device=dev)
        scratch = torch.empty(2 * n + 1, dtype=torch.int32, device=dev)
        _ok("surr_build_csr", lib().surr_build_csr(_p(pairs), int(pairs.shape[0]), n, _p(self.row_ptr),
                                                   _p(self.col), _p(scratch), _stream(torch, dev)))
        self.recv = torch.empty(max(self.n_edges, 1), dtype=torch.int32, device=dev)


class SurrogateNet:
    def __init__(self, device="cuda", seed=2106 + 5000):
        import torch
        self.dev = torch.device(device)
        offs, total = param_layout()
        shapes = [(16, 128), (144, 128), (256, 128), (256, 128), (256, 128), (128, 8)]
        rng = np.random.default_rng(seed)
        p = np.zeros(total, np.float32)
        for (ow, ob), (i, j) in zip(offs, shapes):
            p[ow:ow + i * j] = rng.normal(0.0, math.sqrt(2.0 / i), i * j) * (0.1 if j == 8 else 1.0)
        self.total = total
        self.params = torch.tensor(p, device=self.dev)
        self.pb = torch.empty(total, dtype=torch.bfloat16, device=self.dev)
        self.m = torch.zeros(total, dtype=torch.float32, device=self.dev)
        self.v = torch.zeros(total, dtype=torch.float32, device=self.dev)
        self.grad = torch.zeros(total, dtype=torch.float32, device=self.dev)
        self.step_count = 0
        self.out_scale = torch.ones(6, dtype=torch.float32, device=self.dev)
        self.ws = None
        self.sync_bf16()

    def sync_bf16(self):
        import torch
        _ok("surr_params_to_bf16", lib().surr_params_to_bf16(_p(self.params), _p(self.pb), self.total,
                                                             _stream(torch, self.dev)))

    def _workspace(self, n, ne):
        import torch
        size = C.c_size_t(0)
        _ok("surr_workspace_bytes", lib().surr_workspace_bytes(n, ne, C.byref(size)))
        if self.ws is None or self.ws.numel() < size.value:
            self.ws = torch.empty(int(size.value), dtype=torch.uint8, device=self.dev)
        return self.ws

    def features(self, x, v, w, radius, g: Graph, geom):
        import torch
        X = torch.empty((g.n, 16), dtype=torch.float32, device=self.dev)
        E = torch.empty((max(g.n_edges, 1), 16), dtype=torch.float32, device=self.dev)
        _ok("surr_features", lib().surr_features(_p(x), _p(v), _p(w), _p(radius), g.n, _p(g.row_ptr), _p(g.col),
                                                 g.n_edges, _p(geom), _p(g.recv), _p(X), _p(E),
                                                 _stream(torch, self.dev)))
        return X, E

    def forward(self, X, E, g: Graph):
        import torch
        ws = self._workspace(g.n, g.n_edges)
        Y = torch.empty((g.n, 8), dtype=torch.float32, device=self.dev)
        _ok("surr_forward", lib().surr_forward(_p(self.pb), _p(self.params), _p(X), _p(E), _p(g.row_ptr), _p(g.col),
                                               g.n, g.n_edges, _p(ws), _p(Y), _stream(torch, self.dev)))
        return Y

    def backward(self, dY, g: Graph):
        import torch
        _ok("surr_backward", lib().surr_backward(_p(self.pb), _p(dY), _p(g.row_ptr), _p(g.col), g.n, g.n_edges,
                                                 _p(self.ws), _p(self.grad), _stream(torch, self.dev)))
        return self.grad

    def loss_grad(self, Y, T, weights):
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        dY = torch.empty_like(Y)
        _ok("surr_mse", lib().surr_mse(_p(Y), _p(T), _p(weights), int(Y.shape[0]), _p(loss), _p(dY),
                                       _stream(torch, self.dev)))
        return loss, dY

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        import torch
        self.step_count += 1
        _ok("surr_adam", lib().surr_adam(_p(self.params), _p(self.pb), _p(self.grad), _p(self.m), _p(self.v),
                                         self.total, lr, b1, b2, eps, self.step_count, _stream(torch, self.dev)))

    def train_step(self, X, E, g, T, weights, lr):
        Y = self.forward(X, E, g)
        loss, dY = self.loss_grad(Y, T, weights)
        self.backward(dY, g)
        self.adam(lr)
        return loss

    def apply(self, x, v, w, radius, Y, geom, kdt):
        import torch
        _ok("surr_apply", lib().surr_apply(_p(x), _p(v), _p(w), _p(radius), int(x.shape[0]), _p(Y), _p(geom),
                                           _p(self.out_scale), float(kdt), _stream(torch, self.dev)))


def drum_geometry(wl, device):
    """{cx, y0, cz, Rd, L, d0, vs, 0} of a drum workload (axis along y through the origin)."""
    import torch
    R, L = wl.cfg["drum_radius"], wl.cfg["drum_length"]
    omega = abs(wl.walls[0].get("omega", 1.0)) or 1.0
    d0 = 2.0 * float(wl.radius.max())
    return torch.tensor([0.0, 0.0, 0.0, R, L, d0, omega * R, 0.0], dtype=torch.float64, device=device)
