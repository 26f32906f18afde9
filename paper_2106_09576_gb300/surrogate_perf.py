"""Timing of the surrogate's kernels at the size of the 200,000-sphere drum.

    python -m paper_2106_09576_gb300.surrogate_perf              # JSON line of timings
    python -m paper_2106_09576_gb300.surrogate_perf --forward 3  # only 3 forward passes (for ncu)

Reports, with CUDA events after warm-up:
  - the 128-wide product on its own, C [M][128] = A [M][K] W [K][128] with M = 1,228,800 and
    K = 144 and 256 (BF16 in, FP32 out): the tcgen05 kernel the forward pass uses, the
    mma.sync kernel the backward pass uses, and torch.matmul (cuBLAS, BF16 out) for context;
    bytes = M (2 K + 4 * 128) + 2 K 128;
  - forward and backward passes of the network on the radius-1.2 d graph of the
    200,000-sphere drum fill (about 2.3M directed edges).
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    import torch

    import workloads
    from . import surrogate as SG

    ap = argparse.ArgumentParser()
    ap.add_argument("--forward", type=int, default=0, help="only run this many forward passes")
    a = ap.parse_args()
    dev = torch.device("cuda")
    s = torch.cuda.current_stream()

    def timeit(fn, reps=10, warm=3):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    wl = workloads.drum(n=200_000, precision="mixed", spacing=0.999)
    x = torch.tensor(wl.x, device=dev)
    v = torch.tensor(wl.v, device=dev)
    w = torch.tensor(wl.w, device=dev)
    r = torch.tensor(wl.radius, device=dev)
    net = SG.SurrogateNet()
    t0 = time.perf_counter()
    g = SG.Graph(x, 1.2 * 2.0 * float(wl.radius.max()), wl.cfg["domain_lo"], wl.cfg["domain_hi"])
    torch.cuda.synchronize()
    t_graph = time.perf_counter() - t0
    X, E = net.features(x, v, w, r, g, SG.drum_geometry(wl, dev))
    if a.forward:
        for _ in range(a.forward):
            Y = net.forward(X, E, g)
        torch.cuda.synchronize()
        print(json.dumps({"nodes": g.n, "edges": g.n_edges, "forwards": a.forward, "checksum": float(Y.abs().sum())}))
        return

    out = {"nodes": g.n, "edges": g.n_edges, "graph_s": t_graph}
    out["forward_ms"] = timeit(lambda: net.forward(X, E, g))
    Y = net.forward(X, E, g)
    dY = torch.randn_like(Y)
    out["backward_ms"] = timeit(lambda: net.backward(dY, g))
    fl = 2 * (g.n * 16 * 128 + g.n_edges * 144 * 128 + 3 * g.n * 256 * 128 + g.n * 128 * 8)
    out["forward_gflop"] = fl / 1e9
    del X, E, Y, dY, g

    M, N = 1_228_800, 128
    lib = SG.lib()
    for K in (144, 256):
        A = torch.randn(M, K, device=dev).to(torch.bfloat16)
        B = torch.randn(K, N, device=dev).to(torch.bfloat16)
        C = torch.empty(M, N, device=dev)
        byt = M * K * 2 + K * N * 2 + M * N * 4
        ref = A[:4096].float() @ B.float()
        for name, fn in (("tcgen05", lambda: lib.surr_gemm_bf16_tc(SG._p(A), SG._p(B), SG._p(C), M, K,
                                                                     SG._stream(torch, dev))),
                         ("mma_sync", lambda: lib.surr_gemm_bf16(SG._p(A), SG._p(B), SG._p(C), M, K, N,
                                                                  SG._stream(torch, dev)))):
            ms = timeit(lambda: SG._ok(name, fn()))
            err = float((C[:4096] - ref).abs().max() / ref.abs().max())
            out[f"{name}_K{K}"] = {"ms": ms, "tflops": 2 * M * N * K / ms / 1e9, "gbs": byt / ms / 1e6,
                                   "rel_err": err}
        ms = timeit(lambda: torch.matmul(A, B))
        out[f"cublas_bf16out_K{K}"] = {"ms": ms, "gbs": (M * K * 2 + K * N * 2 + M * N * 2) / ms / 1e6}
        del A, B, C
    print(json.dumps(out))


if __name__ == "__main__":
    main()
