"""Autotuner for the launch and search parameters of a workload: the step-kernel block
size (threads per block), how the mixed-precision step spreads the pairs over its lanes
(pair_eval: each touching pair evaluated once, by the lane of its owner, with the reaction
handed to the partner's lane -- or evaluated by both partners' lanes), and the search
skin (list length vs search frequency).  Each candidate runs the workload's own first
steps in a fresh context and is timed with CUDA events on the context's stream; the
fastest wins.  None of them changes the physics: block size and pair evaluation are
launch choices (the same law on the same pairs; only the order of the FP32 force sums
differs), and any skin finds every contact (a smaller one searches more often)."""
from __future__ import annotations

import itertools


def autotune(wl, precision="mixed", blocks=(64, 128), skin_factors=(0.2, 0.3, 0.45), pair_evals=("once", "both"),
             warmup=100, steps=300, device=None):
    """Returns (overrides, table): `overrides` are the cfg entries of the fastest candidate
    (step_block, pair_eval, skin), `table` lists every candidate with its ms per step."""
    import torch

    from .dem import DEM

    dmax = 2.0 * float(wl.radius.max())
    table = []
    best = None
    for blk, pe, sf in itertools.product(blocks, pair_evals, skin_factors):
        cfg = dict(wl.cfg, step_block=int(blk), pair_eval=pe, skin=float(sf * dmax))
        g = DEM(cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls, precision=precision, device=device)
        g.step(warmup)
        g.sync()
        s = torch.cuda.current_stream(g.device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.step(steps)
        e1.record(s)
        torch.cuda.synchronize(g.device)
        ms = e0.elapsed_time(e1) / steps
        g.close()
        del g
        torch.cuda.empty_cache()
        row = {"step_block": int(blk), "pair_eval": pe, "skin_over_dmax": float(sf), "ms_per_step": ms}
        table.append(row)
        if best is None or ms < best["ms_per_step"]:
            best = row
    return ({"step_block": best["step_block"], "pair_eval": best["pair_eval"], "skin": best["skin_over_dmax"] * dmax},
            table)
