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
              "surr_backward", "surr_mse", "surr_adam", "surr_gemm_bf16", "surr_gemm_bf16_tc", "surr_tc_timeouts", "surr_tc_wait_probe",
              "surr_features", "surr_targets", "surr_apply"]


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
        "surr_gemm_bf16_tc": [P, P, P, I64, I64, P],
        "surr_tc_timeouts": [C.POINTER(C.c_int)],
        "surr_tc_wait_probe": [C.POINTER(C.c_int), C.POINTER(C.c_int)],
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


# ------------------------------------------------------------------ data, training, rollout
class Sample:
    __slots__ = ("graph", "X", "E", "T")

    def __init__(self, graph, X, E, T):
        self.graph, self.X, self.E, self.T = graph, X, E, T


def _state(dem_ctx, n, dev):
    import torch
    x = torch.empty((n, 3), dtype=torch.float64, device=dev)
    v = torch.empty_like(x)
    w = torch.empty_like(x)
    a = torch.empty(n, dtype=torch.uint8, device=dev)
    dem_ctx.state((x, v, w, a))
    return x, v, w


def drum_trajectories(n_traj, n_particles, settle_steps, samples_per_traj, gap_steps, net, device="cuda",
                      seed0=None, omega=1.0, noise_v=0.0, noise_x=0.0):
    """Training samples from DEM runs of small rotating drums (the 200k drum's materials,
    radii and speed, scaled down; seeded per trajectory with seed_for(5, t)).  After
    settling, every gap_steps steps: the graph and features of a state and the increments
    over the next K_STEPS steps.  Targets are scaled by net.out_scale.

    With noise_v > 0 the input velocities and spins are perturbed by Gaussian noise of
    standard deviation noise_v times the velocity scale (spins: divided by the radius), and
    the targets become the increments from the perturbed state to the true one, so the
    network learns to pull a drifting state back; noise_x perturbs the input positions by
    noise_x times the largest diameter (the graph and the features see the perturbed
    positions).  The noise is seeded per trajectory."""
    import torch
    import workloads
    from .dem import DEM
    dev = torch.device(device)
    out = []
    for t in range(n_traj):
        seed = workloads.seed_for(5, t) if seed0 is None else seed0 + t
        wl = workloads.drum(n=n_particles, seed=seed, omega=omega, precision="mixed", spacing=0.999)
        g = DEM(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls, precision="mixed", device=dev)
        r = torch.tensor(wl.radius, device=dev)
        geom = drum_geometry(wl, dev)
        cut = 1.2 * 2.0 * float(wl.radius.max())
        g.step(settle_steps)
        gen = torch.Generator(device=dev)
        gen.manual_seed(seed)
        vs, d0 = float(geom[6]), float(geom[5])
        for _ in range(samples_per_traj):
            x0, v0, w0 = _state(g, wl.n, dev)
            g.step(K_STEPS)
            _, v1, w1 = _state(g, wl.n, dev)
            if noise_v > 0.0:
                v0 = v0 + noise_v * vs * torch.randn(v0.shape, generator=gen, device=dev, dtype=v0.dtype)
                w0 = w0 + noise_v * vs * torch.randn(w0.shape, generator=gen, device=dev, dtype=w0.dtype) / \
                    r.double()[:, None]
            if noise_x > 0.0:
                x0 = x0 + noise_x * d0 * torch.randn(x0.shape, generator=gen, device=dev, dtype=x0.dtype)
            G = Graph(x0, cut, wl.cfg["domain_lo"], wl.cfg["domain_hi"])
            X, E = net.features(x0, v0, w0, r, G, geom)
            T = torch.empty((wl.n, 6), dtype=torch.float32, device=dev)
            _ok("surr_targets", lib().surr_targets(_p(v0), _p(w0), _p(v1), _p(w1), _p(r), wl.n, _p(geom),
                                                   _p(net.out_scale), _p(T), _stream(torch, dev)))
            out.append(Sample(G, X, E, T))
            g.step(gap_steps)
        g.close()
    return out


def fit_output_scale(net, samples):
    """Per-output scale = RMS of the (unscaled) targets, so every output has unit size."""
    import torch
    T = torch.cat([s.T for s in samples]) * net.out_scale
    sc = torch.sqrt((T.double() ** 2).mean(0)).float().clamp_min(1e-12)
    for s in samples:
        s.T.mul_(net.out_scale / sc)
    net.out_scale = sc


def train(net, samples, epochs, lr=1e-3, seed=0):
    import torch
    w = torch.ones(6, dtype=torch.float32, device=net.dev)
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        tot = torch.zeros(1, dtype=torch.float32, device=net.dev)
        for k in rng.permutation(len(samples)):
            s = samples[k]
            tot += net.train_step(s.X, s.E, s.graph, s.T, w, lr)
        hist.append(float(tot.item()) / len(samples))
    return hist


def evaluate(net, samples):
    """(MSE of the network, MSE of predicting no change) over samples, scaled targets."""
    import torch
    w = torch.ones(6, dtype=torch.float32, device=net.dev)
    a = b = 0.0
    for s in samples:
        Y = net.forward(s.X, s.E, s.graph)
        loss, _ = net.loss_grad(Y, s.T, w)
        a += float(loss.item())
        b += float((s.T.double() ** 2).mean().item())
    return a / len(samples), b / len(samples)


def rollout(net, wl, dem_ctx, n_equiv_steps, max_overlap=0.02, max_ke_gain=0.2, overlap_factor=0.0,
            device="cuda", stats=None):
    """Advances the drum by n_equiv_steps DEM-step equivalents with the surrogate (K_STEPS
    per network evaluation), starting from dem_ctx's current state.  Each surrogate step is
    checked on the state it produces: if the largest particle-particle overlap exceeds the
    limit (max_overlap of the largest diameter, or overlap_factor times the largest overlap
    of the last state plain DEM produced, whichever is larger), or the kinetic energy
    (translation and spin) exceeds by more than max_ke_gain the energy of that DEM state
    (the start, or the last fallback), the step is discarded and the K_STEPS are taken by
    plain DEM from the previous state instead (fallback).  Returns the final state, the
    number of fallbacks and of surrogate steps; `stats` (a dict), if given, receives the
    rejections by cause and the mean largest overlap of the DEM states."""
    import torch
    dev = torch.device(device)
    x, v, w = _state(dem_ctx, wl.n, dev)
    r = torch.tensor(wl.radius, device=dev)
    m = torch.tensor(wl.cfg["density"] * 4.0 / 3.0 * np.pi * wl.radius.astype(np.float64) ** 3, device=dev)
    geom = drum_geometry(wl, dev)
    d0 = 2.0 * float(wl.radius.max())
    cut = 1.2 * d0
    kdt = K_STEPS * wl.cfg["dt"]
    lo, hi = wl.cfg["domain_lo"], wl.cfg["domain_hi"]

    inertia = 0.4 * m * r.double() ** 2

    def ke(v_, w_):
        return float((0.5 * m * (v_ * v_).sum(1) + 0.5 * inertia * (w_ * w_).sum(1)).sum().item())

    def largest_overlap(x_, v_, w_, G_):
        if not G_.n_edges:
            return 0.0
        _, E_ = net.features(x_, v_, w_, r, G_, geom)
        return 0.01 * float(E_[: G_.n_edges, 4].max().item())   # in d0

    fall = surr = rej_ovl = rej_ke = 0
    G = Graph(x, cut, lo, hi)
    ke_ref = ke(v, w)
    ovl_ref = largest_overlap(x, v, w, G)
    ovl_sum, ovl_n = ovl_ref, 1
    for _ in range(n_equiv_steps // K_STEPS):
        X, E = net.features(x, v, w, r, G, geom)
        Y = net.forward(X, E, G)
        x1, v1, w1 = x.clone(), v.clone(), w.clone()
        net.apply(x1, v1, w1, r, Y, geom, kdt)
        G1 = Graph(x1, cut, lo, hi)
        ovl = largest_overlap(x1, v1, w1, G1)
        k1 = ke(v1, w1)
        ovl_ok = ovl <= max(max_overlap, overlap_factor * ovl_ref)
        ke_ok = k1 == k1 and k1 <= ke_ref * (1.0 + max_ke_gain) + 1e-12
        if ovl_ok and ke_ok:
            x, v, w, G = x1, v1, w1, G1
            surr += 1
            continue
        rej_ovl += 0 if ovl_ok else 1
        rej_ke += 0 if ke_ok else 1
        dem_ctx.set_state(x, v, w)
        dem_ctx.step(K_STEPS)
        x, v, w = _state(dem_ctx, wl.n, dev)
        G = Graph(x, cut, lo, hi)
        ke_ref = ke(v, w)
        ovl_ref = largest_overlap(x, v, w, G)
        ovl_sum += ovl_ref
        ovl_n += 1
        fall += 1
    if stats is not None:
        stats.update(rejected_overlap=rej_ovl, rejected_energy=rej_ke, dem_mean_largest_overlap=ovl_sum / ovl_n)
    return (x, v, w), fall, surr
