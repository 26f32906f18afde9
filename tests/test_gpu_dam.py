"""The dam break (the paper's weak-scaling case): the FP64 path equals the oracle bit for
bit through the removal of the dam, and the mixed path's collapse front follows the FP64
path's (macroscopic comparison of a chaotic flow)."""
import numpy as np
import pytest

import workloads
from gpu_helpers import make_gpu, make_oracle
from test_gpu_parity import compare_exact

pytestmark = pytest.mark.gpu


def test_dam_break_fp64_equals_oracle_through_the_removal():
    wl = workloads.dam_break(n=2000, seed=5, length=0.06, height=0.08, t_dam=0.004, precision="fp64")
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    for chunk in (500, 500, 3000, 6000):          # the dam goes at step 1000
        g.step(chunk)
        o.step(chunk)
        compare_exact(g, o)
    x, _, _, _ = g.state()
    assert x[:, 0].max() > 0.03                    # spheres have crossed the dam line


def front(x, d):
    """x position of the collapse front: 99th percentile of x."""
    return float(np.quantile(x[:, 0], 0.99))


def test_dam_break_front_mixed_vs_fp64():
    fronts = {}
    for prec in ("fp64", "mixed"):
        wl = workloads.dam_break(n=20000, seed=7, length=0.12, height=0.12, t_dam=0.02, precision=prec,
                                 depth=0.012)
        g = make_gpu(wl, prec)
        g.step(5000)                               # settling behind the dam until it goes
        out = []
        for _ in range(4):
            g.step(6000)
            x, _, _, _ = g.state()
            out.append(front(x, 1e-3))
        fronts[prec] = np.array(out)
        g.close()
    print("front fp64", fronts["fp64"], "mixed", fronts["mixed"])
    assert fronts["fp64"][-1] > max(fronts["fp64"][0], 0.06) + 5e-3   # the front runs past the dam line
    assert np.abs(fronts["mixed"] - fronts["fp64"]).max() <= 3e-3   # within 3 d
