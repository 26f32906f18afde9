"""The paper's other options on the GPU: the linear contact model, viscous rolling,
explicit Euler and translating walls.  The FP64 path reproduces the oracle bit for bit
(same operations in the same order); the mixed path stays within the same tolerance as
the default model."""
import numpy as np
import pytest

import workloads
from gpu_helpers import force_error, make_gpu, make_oracle, masses, torque_error
from test_gpu_parity import MIXED_TOL, compare_exact, dense, with_history

pytestmark = pytest.mark.gpu

VARIANTS = {
    "linear": dict(contact_model=1, linear_velocity=0.7),
    "viscous-rolling": dict(rolling_model=2),
    "euler": dict(integrator=1),
    "linear+viscous+euler": dict(contact_model=1, linear_velocity=0.4, rolling_model=2, integrator=1),
}


def with_variant(wl, **kw):
    wl.cfg.update(kw)
    for m in (wl.cfg["particle"], wl.cfg["wall"]):
        if kw.get("rolling_model") == 2:
            m["mu_roll"] = 0.5                     # s/m for the viscous model
    return wl


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_fp64_bit_exact_with_rebuilds(name):
    wl = with_variant(dense(n=1500, seed=61, speed=1.0), **VARIANTS[name])
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    with_history(wl, g, o)
    Fg, Mg = g.forces()
    Fo, Mo = o.forces()
    assert np.array_equal(Fg, Fo) and np.array_equal(Mg, Mo)
    for chunk in (1, 20, 180):
        g.step(chunk)
        o.step(chunk)
        compare_exact(g, o)
    assert g.stats()["rebuilds"] == o.stats()["rebuilds"] >= 2


def piston(n=1200, precision="fp64", U=0.05):
    """A lattice in a box whose lid descends at U and whose floor slides sideways."""
    wl = dense(n=n, seed=71, speed=0.2)
    L = float(wl.x[:, 2].max() + wl.radius.max() + 1e-4)     # the lid touches after ~2 ms
    walls = [w for w in wl.walls if not (w["normal"][2] != 0.0)]
    walls.append(workloads.plane((0, 0, 0), (0, 0, 1), velocity=(0.02, 0.0, 0.0)))
    walls.append(workloads.plane((0, 0, L), (0, 0, -1), velocity=(0.0, 0.0, -U), translates=1))
    wl.walls = walls
    return wl


def test_translating_lid_fp64_bit_exact():
    wl = piston()
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    for chunk in (50, 450, 500):
        g.step(chunk)
        o.step(chunk)
        compare_exact(g, o)
    assert g.stats()["n_wall_touch"] > 0


def test_translating_lid_mixed_follows_fp64():
    wl = piston(precision="mixed")
    gm, gf = make_gpu(wl, "mixed"), make_gpu(wl, "fp64")
    gm.step(300)
    gf.step(300)
    xm, _, _, _ = gm.state()
    xf, _, _, _ = gf.state()
    assert np.abs(xm - xf).max() < 1e-7
    assert gm.stats()["n_wall_touch"] == gf.stats()["n_wall_touch"] > 0


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_mixed_one_step_within_tolerance(name):
    wl = with_variant(dense(n=2000, seed=81), **VARIANTS[name])
    g, o = make_gpu(wl, "mixed"), make_oracle(wl)
    with_history(wl, g, o)
    Fg, Mg = g.forces()
    Fo, Mo = o.forces()
    Fa, Ma = o.force_scales()
    m = masses(wl)
    gvec = wl.cfg["gravity"]
    ef = force_error(Fg, Fo, Fa, m, gvec)
    em = torque_error(Mg, Mo, Ma, m, wl.radius.astype(float), gvec)
    print(f"{name}: mixed one-step relative error force {ef:.3e} torque {em:.3e}")
    assert ef <= MIXED_TOL and em <= MIXED_TOL
    g.step(20)
    o.step(20)
    xg, _, _, ag = g.state()
    xo, _, _, ao = o.state()
    assert np.array_equal(ag, ao)
    assert np.abs(xg - xo).max() < 1e-9
