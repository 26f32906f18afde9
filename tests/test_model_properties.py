"""Properties of the method itself that bound what any implementation can reproduce.

The constant rolling-resistance model (Table rolling_torque) applies a torque of full
magnitude mu_r R_e |F_n| in the direction of w_i - w_j for any non-zero relative spin.
Starting from rest, the relative spin is pure rounding noise, and the model turns it into
spins of order 1e-3..1e-2 rad/s within a few steps.  Two correct evaluations that round
differently (FP64 vs FP32 contact arithmetic) therefore disagree on spins from rest;
comparisons of the mixed path are made from states with non-zero spins.
"""
import numpy as np

import oracle
import workloads


def _spin_spread(rolling):
    wl = workloads.drum(n=3000, seed=2002, omega=1.0, spacing=0.999)
    wl.cfg["rolling_model"] = rolling
    a = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
    b = oracle.OracleSim(wl.cfg, np.nextafter(wl.x, np.inf), wl.v, wl.w, wl.radius, wl.walls)
    a.step(4)
    b.step(4)
    _, _, wa, _ = a.state()
    _, _, wb, _ = b.state()
    assert a.stats()["n_touch"] > 0
    return np.abs(wa - wb).max()


def test_constant_rolling_model_amplifies_rounding_noise_from_rest():
    with_rolling = _spin_spread(1)
    without = _spin_spread(0)
    assert without < 1e-12            # one ulp of position stays one-ulp-sized
    assert with_rolling > 1e-5        # ... unless the rolling torque acts on noise
    assert with_rolling > 1e6 * without
