"""Long rollouts compared on macroscopic quantities.

Trajectories of a granular flow diverge chaotically, so beyond a few thousand steps the
mixed-precision path is compared with the FP64 path through what an experiment would
measure: the discharge rate of a silo (linear fit between 20 % and 80 % discharged), the
packing fraction of the settled bed, and the dynamic angle of repose in a rotating drum,
each averaged over three seeded instances.  The FP64 path itself reproduces the oracle
bit for bit, which the first test checks over a whole discharge."""
import numpy as np
import pytest

import workloads
from gpu_helpers import make_gpu, make_oracle
from macro import angle_of_repose, discharge_rate, packing_fraction

pytestmark = pytest.mark.gpu

D = 3e-3


def mini_silo(n, seed, R, orifice, t_open, height, precision):
    return workloads.silo(n=n, seed=seed, d=D, R=R, orifice=orifice, height=height, t_open=t_open,
                          z_sink=-0.02, precision=precision)


def discharge(sim, wl, settle_steps, chunk, max_steps, stop_fraction=0.81):
    """Steps sim through settling and discharge; returns (times, discharged counts, state at
    the opening of the orifice)."""
    dt = wl.cfg["dt"]
    sim.step(settle_steps)
    opened = sim.state()
    t, out = [], []
    steps = settle_steps
    while steps < max_steps:
        sim.step(chunk)
        steps += chunk
        t.append(steps * dt)
        out.append(wl.n - sim.stats()["n_active"])
        if out[-1] >= stop_fraction * wl.n:
            break
    return np.array(t), np.array(out), opened


def test_silo_discharge_fp64_equals_oracle_to_the_last_particle():
    # a shallow bed: its flat bottom keeps a dead zone, so only about two thirds leave
    wl = mini_silo(1500, 4101, R=0.025, orifice=0.0135, t_open=0.05, height=0.05, precision="fp64")
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    tg, dg, _ = discharge(g, wl, 5000, 1000, 50000, stop_fraction=1.0)
    to, do, _ = discharge(o, wl, 5000, 1000, 50000, stop_fraction=1.0)
    assert np.array_equal(tg, to) and np.array_equal(dg, do)
    for a, b in zip(g.state(), o.state()):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    assert dg[-1] >= 0.5 * wl.n
    rate = discharge_rate(tg, dg, wl.n, lo=0.1, hi=0.5)
    print(f"1500-sphere silo: {rate:.0f} spheres/s through a {2 * 13.5 / 3:.0f} d orifice, "
          f"{dg[-1]} discharged in {tg[-1]:.2f} s")


def test_silo_discharge_rate_and_packing_mixed_vs_fp64():
    rates = {"fp64": [], "mixed": []}
    phis = {"fp64": [], "mixed": []}
    for seed in (4201, 4202, 4203):
        for prec in ("fp64", "mixed"):
            wl = mini_silo(8000, seed, R=0.03, orifice=0.016, t_open=0.08, height=0.13, precision=prec)
            g = make_gpu(wl, prec)
            t, dcount, opened = discharge(g, wl, 8000, 1000, 150000)
            assert dcount[-1] >= 0.8 * wl.n, (prec, seed, dcount[-1])
            rates[prec].append(discharge_rate(t, dcount, wl.n))
            x, _, _, act = opened
            phis[prec].append(packing_fraction(x, wl.radius, act, 0.03, 0.0, D))
            g.close()
    rf, rm = np.mean(rates["fp64"]), np.mean(rates["mixed"])
    pf, pm = np.mean(phis["fp64"]), np.mean(phis["mixed"])
    print(f"discharge rate fp64 {rates['fp64']} mixed {rates['mixed']}: {abs(rm - rf) / rf:.4f} relative")
    print(f"packing fraction fp64 {phis['fp64']} mixed {phis['mixed']}: {abs(pm - pf):.5f}")
    assert abs(rm - rf) <= 0.03 * rf
    assert abs(pm - pf) <= 0.005
    assert 0.5 < pf < 0.66


def test_drum_dynamic_angle_of_repose_mixed_vs_fp64():
    # Each precision's angle is one draw of a chaotic flow: two realizations per seed (the
    # second with the initial positions moved by up to 1 nm) so that the comparison has
    # six samples a side; one sample per seed gave offsets of 1-1.5 degrees by chance.
    angles = {"fp64": [], "mixed": []}
    for seed in (4301, 4302, 4303):
        for prec in ("fp64", "mixed"):
            for rep in range(2):
                wl = workloads.drum(n=2500, seed=seed, omega=3.0, precision=prec)
                wl.cfg["dt"] = 1e-5
                if rep:
                    wl.x = wl.x + np.random.default_rng(rep).uniform(-1e-9, 1e-9, wl.x.shape)
                g = make_gpu(wl, prec)
                g.step(30000)
                samples = []
                for _ in range(10):
                    g.step(3000)
                    x, _, _, act = g.state()
                    samples.append(angle_of_repose(x, wl.radius, act, wl.cfg["drum_length"],
                                                   2 * float(wl.radius.max())))
                angles[prec].append(float(np.mean(samples)))
                g.close()
    af, am = np.array(angles["fp64"]), np.array(angles["mixed"])
    se = np.sqrt(af.var(ddof=1) / len(af) + am.var(ddof=1) / len(am))
    print(f"dynamic angle of repose fp64 {af} mixed {am} (deg); standard error {se:.3f}")
    assert abs(am.mean() - af.mean()) <= max(1.0, 2.0 * se)
    assert 10.0 < af.mean() < 50.0
