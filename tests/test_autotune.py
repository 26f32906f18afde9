"""Host logic of the autotuner, on CPU: every (block size, pair evaluation, skin) candidate is timed once on
the workload in a fresh context, and the fastest one's settings come back as overrides.
The contexts and CUDA events are stand-ins that report a chosen time per candidate."""
import numpy as np
import pytest

import workloads
from paper_2106_09576_gb300 import autotune as A
from paper_2106_09576_gb300 import dem as D


def test_autotuner_times_every_candidate_and_returns_the_fastest(monkeypatch):
    import torch

    wl = workloads.lattice(n=64, seed=1)
    dmax = 2.0 * float(wl.radius.max())
    # ms per step for each candidate: block 128, both sides, skin 0.3 d is the fastest
    base = {(64, 0.2): 3.0, (64, 0.3): 2.5, (64, 0.45): 2.8, (128, 0.2): 2.2, (128, 0.3): 1.9, (128, 0.45): 2.4}
    cost = {}
    for (b, sf), c in base.items():
        cost[(b, "once", sf)] = c + 0.3
        cost[(b, "both", sf)] = c
    made = []
    clock = {"t": 0.0}

    class FakeDEM:
        def __init__(self, cfg, x, v, w, radius, walls, precision=None, device=None):
            self.key = (cfg["step_block"], cfg["pair_eval"], round(cfg["skin"] / dmax, 6))
            self.device = "cpu"
            made.append(self.key)

        def step(self, n):
            clock["t"] += cost[self.key] * n

        def sync(self):
            pass

        def close(self):
            pass

    class FakeEvent:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = clock["t"]

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(D, "DEM", FakeDEM)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda device=None: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda device=None: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    over, table = A.autotune(wl, warmup=10, steps=100)
    assert sorted(made) == sorted(cost)                       # one fresh context per candidate
    assert len(table) == 12
    for row in table:
        assert row["ms_per_step"] == pytest.approx(cost[(row["step_block"], row["pair_eval"], row["skin_over_dmax"])])
    assert over["step_block"] == 128 and over["pair_eval"] == "both" and over["skin"] == pytest.approx(0.3 * dmax)
    assert np.isfinite([r["ms_per_step"] for r in table]).all()
