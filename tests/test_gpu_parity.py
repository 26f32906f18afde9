"""Parity of the CUDA library (through its C ABI) with the CPU oracle on seeded inputs.

FP64 path: the library evaluates every pair term with the oracle's operations, in the
oracle's order, and sums each particle's contacts in partner-id order, so its results
must be bit-identical to the oracle's: pair sets, forces, positions, velocities,
tangential overlaps and active flags, over many steps with rebuilds.

Mixed path: forces within 1e-5 of the oracle's, relative to the particle's contact-force
scale (sum of |contact force| + m|g|), which keeps cancelling net forces from dominating.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import (force_error, make_gpu, make_oracle, masses, random_history, torque_error,
                         touching_pairs)

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


def free_box(n, seed, L=0.03):
    """Uniform random centres (overlaps allowed) plus adversarial pairs at the
    search threshold and one ulp either side."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, (n, 3))
    R = rng.uniform(0.5e-3, 1e-3, n).astype(np.float32)
    rc = 1.3 * 2 * float(R.max())
    for k, f in enumerate([1.0, 1.0 - 2 ** -52, 1.0 + 2 ** -52, 1.0 - 2 ** -50, 1.0 + 2 ** -50]):
        x[2 * k + 1] = x[2 * k] + np.array([rc * f, 0.0, 0.0])
    cfg = dict(density=2500.0, particle=workloads.material(), wall=workloads.material(),
               gravity=(0, 0, 0), dt=1e-6, neighbor_factor=1.3, domain_lo=(0, 0, 0),
               domain_hi=(L, L, L))
    return workloads.Workload("free", cfg, [], x, np.zeros((n, 3)), np.zeros((n, 3)), R)


def numpy_pairs(x, rc):
    out = []
    for i in range(len(x)):
        d = x[i + 1:] - x[i]
        s = d[:, 0] * d[:, 0]
        s = s + d[:, 1] * d[:, 1]
        s = s + d[:, 2] * d[:, 2]
        out.extend((i, j) for j in np.nonzero(s < rc * rc)[0] + i + 1)
    return np.array(out, dtype=np.int32).reshape(-1, 2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pair_sets_bit_exact(precision, seed):
    wl = free_box(1500, seed)
    g = make_gpu(wl, precision)
    o = make_oracle(wl)
    ref = numpy_pairs(wl.x, 1.3 * 2 * float(wl.radius.max()))
    got = g.pairs()
    assert np.array_equal(got, ref)
    assert np.array_equal(o.pairs(), ref)


def dense(n=1000, seed=21, poly=0.1, speed=0.5, spin=50.0):
    """Jittered lattice at the mean diameter: about half of the neighbours overlap."""
    wl = workloads.lattice(n=n, seed=seed, spacing=1.0 - 0.5 * poly, jitter=0.004, speed=speed, spin=spin,
                           poly=poly)
    return wl


def with_history(wl, g, o, seed=5):
    tp = touching_pairs(wl.x, wl.radius.astype(np.float64))
    p, vals = random_history(wl, tp, seed)
    rng = np.random.default_rng(seed + 1)
    dtw = rng.normal(0, 2e-6, (wl.n, len(wl.walls), 3)) * (rng.random((wl.n, len(wl.walls), 1)) < 0.2)
    g.set_history(p, vals, dtw)
    o.set_history(p, vals, dtw)
    return p


@pytest.mark.parametrize("n", [1, 2, 129, 1000, 5003])
def test_initial_forces_fp64_bit_exact(n):
    wl = dense(n=n, seed=100 + n)
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    if n > 2:
        with_history(wl, g, o)
    Fg, Mg = g.forces()
    Fo, Mo = o.forces()
    assert np.array_equal(Fg, Fo)
    assert np.array_equal(Mg, Mo)
    if n >= 129:
        assert o.stats()["n_touch"] > n // 4      # the lattice is dense: many contacts


def compare_exact(g, o):
    xg, vg, wg, ag = g.state()
    xo, vo, wo, ao = o.state()
    assert np.array_equal(ag, ao)
    assert np.array_equal(xg, xo)
    assert np.array_equal(vg, vo)
    assert np.array_equal(wg, wo)
    Fg, Mg = g.forces()
    Fo, Mo = o.forces()
    assert np.array_equal(Fg, Fo) and np.array_equal(Mg, Mo)
    pg, hg, wg_ = g.history()
    po, ho, wo_ = o.history()
    assert np.array_equal(pg, po) and np.array_equal(hg, ho)
    assert np.array_equal(wg_, wo_)


@pytest.mark.parametrize("n", [1000, 5003])
def test_steps_fp64_bit_exact_with_rebuilds(n):
    wl = dense(n=n, seed=7, speed=1.0)
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    with_history(wl, g, o)
    for chunk in (1, 9, 90, 200):
        g.step(chunk)
        o.step(chunk)
        compare_exact(g, o)
    sg, so = g.stats(), o.stats()
    assert sg["rebuilds"] == so["rebuilds"] and sg["rebuilds"] >= 3
    assert sg["n_pairs"] == so["n_pairs"] and sg["n_touch"] == so["n_touch"]
    assert sg["n_wall_touch"] == so["n_wall_touch"] and sg["steps"] == so["steps"]


def small_drum(n=3000, precision="fp64"):
    # FCC at 0.999 d_max: the largest neighbours touch from the start
    return workloads.drum(n=n, seed=2002, omega=3.0, precision=precision, spacing=0.999)


def small_silo(n=2500, precision="fp64", t_open=2e-3):
    wl = workloads.silo(n=n, seed=3003, d=5e-3, R=0.04, orifice=0.012, height=0.2, t_open=t_open,
                        precision=precision)
    wl.cfg["z_sink"] = -0.02
    wl.cfg["domain_lo"] = (-0.04, -0.04, -0.03)
    return wl


def test_drum_fp64_bit_exact():
    wl = small_drum()
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    for chunk in (500, 2500):
        g.step(chunk)
        o.step(chunk)
        compare_exact(g, o)
    st = g.stats()
    assert st["n_wall_touch"] > 0 and st["n_touch"] > 0


def test_silo_discharge_fp64_bit_exact():
    wl = small_silo()
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    for _ in range(6):
        g.step(2000)
        o.step(2000)
    compare_exact(g, o)
    sg = g.stats()
    assert sg["n_active"] == o.stats()["n_active"]
    assert sg["n_active"] < wl.n            # some particles have left through the orifice


def test_constant_search_mode_fp64_bit_exact():
    wl = dense(n=1000, seed=9, speed=0.5)
    wl.cfg["rebuild_every"] = 20
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    g.step(150)
    o.step(150)
    compare_exact(g, o)
    assert g.stats()["rebuilds"] == o.stats()["rebuilds"] == 1 + 150 // 20


def test_set_state_midway_fp64_bit_exact():
    wl = dense(n=1000, seed=13, speed=0.5)
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    g.step(50)
    o.step(50)
    x, v, w, a = o.state()
    v2 = v * 0.5
    a2 = a.copy()
    a2[:10] = False
    g.set_state(v=v2, active=a2)
    o.set_state(v=v2, active=a2.astype(np.uint8))
    g.step(60)
    o.step(60)
    compare_exact(g, o)


def test_eager_launch_equals_graph_launch():
    wl = dense(n=1000, seed=17, speed=1.0)
    g1 = make_gpu(wl, "fp64")
    os.environ["DEM_GB300_EAGER"] = "1"
    try:
        g2 = make_gpu(wl, "fp64")
    finally:
        del os.environ["DEM_GB300_EAGER"]
    g1.step(120)
    g2.step(120)
    s1, s2 = g1.state(), g2.state()
    for a, b in zip(s1, s2):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("maker", ["dense", "drum", "silo"])
@pytest.mark.parametrize("pair_eval", ["once", "both"])
def test_mixed_one_step_forces_within_tolerance(maker, pair_eval):
    if maker == "dense":
        wl = dense(n=2000, seed=31)
    elif maker == "drum":
        wl = workloads.drum(n=3000, seed=2002, omega=3.0, precision="mixed", spacing=0.999)
    else:
        wl = workloads.silo(n=2500, seed=3003, R=0.04, orifice=0.012, height=0.2, precision="mixed",
                            spacing=0.995, jitter=0.002)
    wl.cfg["pair_eval"] = pair_eval
    g, o = make_gpu(wl, "mixed"), make_oracle(wl)
    if maker == "dense":
        with_history(wl, g, o)
    Fg, Mg = g.forces()
    Fo, Mo = o.forces()
    Fa, Ma = o.force_scales()
    m = masses(wl)
    gvec = wl.cfg["gravity"]
    ef = force_error(Fg, Fo, Fa, m, gvec)
    em = torque_error(Mg, Mo, Ma, m, wl.radius.astype(float), gvec)
    print(f"mixed ({pair_eval}) one-step relative error: force {ef:.3e}, torque {em:.3e}")
    assert ef <= MIXED_TOL and em <= MIXED_TOL
    assert Fa.sum() > 0
    # one step later positions and velocities differ by the force error integrated over dt
    g.step(1)
    o.step(1)
    xg, vg, _, ag = g.state()
    xo, vo, _, ao = o.state()
    assert np.array_equal(ag, ao)
    dt = wl.cfg["dt"]
    a_scale = float(np.max(Fa / m)) + float(np.linalg.norm(gvec))
    assert np.abs(xg - xo).max() <= MIXED_TOL * a_scale * dt * dt
    assert np.abs(vg - vo).max() <= 2 * MIXED_TOL * a_scale * dt


def test_mixed_short_rollout_stays_close():
    wl = dense(n=1000, seed=41, speed=0.5)
    g, o = make_gpu(wl, "mixed"), make_oracle(wl)
    g.step(200)
    o.step(200)
    xg, vg, _, _ = g.state()
    xo, vo, _, _ = o.state()
    assert np.abs(xg - xo).max() < 1e-8
    assert np.array_equal(g.pairs(), o.pairs())


def test_history_round_trip_resumes_bit_exact():
    # each path saves and restores its own state and overlaps, then both continue
    wl = dense(n=1000, seed=51, speed=0.5)
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    g.step(100)
    o.step(100)
    xg, vg, wg, ag = g.state()
    pg, hg, hwg = g.history()
    g2 = make_gpu(wl, "fp64")
    g2.set_state(xg, vg, wg, ag)
    g2.set_history(pg, hg, hwg)
    xo, vo, wo, ao = o.state()
    po, ho, hwo = o.history()
    o2 = make_oracle(wl)
    o2.set_state(xo, vo, wo, ao.astype(np.uint8))
    o2.set_history(po, ho, hwo)
    g2.step(40)
    o2.step(40)
    compare_exact(g2, o2)


def test_capacity_error_is_reported():
    wl = dense(n=800, seed=61)
    wl.cfg["neighbor_factor"] = 4.0       # far more than 56 entries per particle
    g = make_gpu(wl, "fp64")
    from paper_2106_09576_gb300 import DemError
    g.step(1)
    with pytest.raises(DemError) as e:
        g.sync()
    assert e.value.code == 3
    with pytest.raises(DemError):
        g.step(1)                        # sticky until the state is set again


def crowded_sphere(k, seed=81):
    """One sphere of radius 5 mm with k spheres of radius 1 mm on its surface (Fibonacci
    directions, each overlapping it by 2 % of the small radius; at k <= 33 the small spheres
    are more than 3 mm apart, so none touches another): the big sphere holds k contacts at
    once.  Random velocities and spins give every pair a tangential overlap."""
    Rb, r = 5e-3, 1e-3
    c = np.array([0.05, 0.05, 0.05])
    t = np.arange(k) + 0.5
    phi = np.arccos(1.0 - 2.0 * t / k)
    th = np.pi * (1.0 + 5.0 ** 0.5) * t
    u = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    x = np.vstack([c, c + (Rb + r - 0.02 * r) * u])
    R = np.array([Rb] + [r] * k, dtype=np.float32)
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, 0.02, (k + 1, 3))
    w = rng.normal(0.0, 2.0, (k + 1, 3))
    cfg = dict(density=2500.0, particle=workloads.material(), wall=workloads.material(),
               gravity=(0, 0, 0), dt=1e-6, neighbor_factor=1.3, domain_lo=(0, 0, 0),
               domain_hi=(0.1, 0.1, 0.1))
    return workloads.Workload("crowded", cfg, [], x, v, w, R)


def test_sphere_holding_every_contact_slot():
    # 32 simultaneous contacts: every slot of the compact overlap list (and, in the mixed
    # path, of the inner list) is in use.  FP64: bit-exact with the oracle over 50 steps.
    # Mixed, both pair evaluations: forces and torques of the first evaluation (tangential
    # overlaps on every pair) within tolerance, positions after 50 steps close, no capacity
    # error.  Later torques are not compared: at these sizes the constant rolling
    # resistance stops a small sphere's relative spin within a few steps (its torque turns
    # the spin by ~0.4 rad/s per step), after which the torque's direction follows the
    # sign of a vanishing relative spin in either precision.
    wl = crowded_sphere(32)
    d = wl.x[1:] - wl.x[1:, None]
    assert np.sqrt((d ** 2).sum(-1) + np.eye(32)).min() > 3e-3
    g, o = make_gpu(wl, "fp64"), make_oracle(wl)
    g.step(50)
    o.step(50)
    compare_exact(g, o)
    assert o.stats()["n_touch"] == 32
    for pair_eval in ("once", "both"):
        wm = crowded_sphere(32)
        wm.cfg["pair_eval"] = pair_eval
        gm, om = make_gpu(wm, "mixed"), make_oracle(wm)
        tp = touching_pairs(wm.x, wm.radius.astype(np.float64))
        assert len(tp) == 32
        p, vals = random_history(wm, tp, 7, frac=1.0)
        gm.set_history(p, vals)
        om.set_history(p, vals)
        Fg, Mg = gm.forces()
        Fo, Mo = om.forces()
        Fa, Ma = om.force_scales()
        m = masses(wm)
        ef = force_error(Fg, Fo, Fa, m, wm.cfg["gravity"])
        em = torque_error(Mg, Mo, Ma, m, wm.radius.astype(float), wm.cfg["gravity"])
        print(f"32 contacts, mixed ({pair_eval}), first evaluation: force {ef:.3e} torque {em:.3e}")
        assert ef <= MIXED_TOL and em <= MIXED_TOL
        gm.step(50)
        om.step(50)
        dx = np.abs(gm.state()[0] - om.state()[0]).max()
        print(f"32 contacts, mixed ({pair_eval}), after 50 steps: max position difference {dx:.3e} m")
        assert dx < 1e-7                    # a lost contact would move a sphere by ~5e-6 m
        assert gm.stats()["n_touch"] == 32
        gm.sync()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_contact_more_than_the_slots_is_a_capacity_error(precision):
    from paper_2106_09576_gb300 import DemError
    g = make_gpu(crowded_sphere(33), precision)
    g.step(1)
    with pytest.raises(DemError) as e:
        g.sync()
    assert e.value.code == 3


def test_nonfinite_and_overlap_errors_are_reported():
    from paper_2106_09576_gb300 import DemError
    wl = dense(n=500, seed=71)
    g = make_gpu(wl, "fp64")
    x = wl.x.copy()
    x[3, 0] = np.nan
    g.set_state(x=x)
    g.step(2)
    with pytest.raises(DemError) as e:
        g.sync()
    assert e.value.code == 4
    g.set_state(x=wl.x)                  # clears the sticky error
    g.step(1)
    g.sync()
    wl.cfg["max_overlap_ratio"] = 1e-6
    g2 = make_gpu(wl, "fp64")
    g2.step(1)
    with pytest.raises(DemError) as e:
        g2.sync()
    assert e.value.code == 5


def search_radius(wl):
    d = 2 * float(wl.radius.max())
    skin = wl.cfg.get("skin", 0.0)
    return d + skin if skin > 0 else wl.cfg["neighbor_factor"] * d


def sampled_parity(wl, precision, steps, n_regions=6, per_region=30, seed=0):
    """Full-size workload from the generator, advanced by dem_step(steps) as the benchmark
    does.  The oracle advances the same generator input restricted to the neighbourhood of
    sampled particles; the neighbourhood has a halo of (steps + 1) search radii, so
    within `steps` steps nothing outside it can reach a sampled particle, and the sampled
    particles' trajectories must agree (bitwise in FP64)."""
    from scipy.spatial import cKDTree
    g = make_gpu(wl, precision)
    pairs0 = g.pairs()                      # contact list of the initial search
    g.step(steps)
    xg, vg, wg, ag = g.state()
    Fg, Mg = g.forces()
    rc = search_radius(wl)
    tree = cKDTree(wl.x)
    rng = np.random.default_rng(seed)
    centres = wl.x[rng.choice(wl.n, n_regions, replace=False)]
    sample = np.unique(np.concatenate([tree.query(c, per_region)[1] for c in centres]))
    halo = (steps + 1) * rc * 1.001
    idx = np.unique(np.concatenate([np.asarray(tree.query_ball_point(wl.x[s], halo), dtype=np.int64)
                                    for s in sample]))
    lut = np.full(wl.n, -1, dtype=np.int64)
    lut[idx] = np.arange(len(idx))
    sub = workloads.Workload("sub", dict(wl.cfg), wl.walls, wl.x[idx], wl.v[idx], wl.w[idx], wl.radius[idx])
    o = make_oracle(sub)
    # pair sets of the sampled particles at the initial search: bit-exact
    insample = np.zeros(wl.n, dtype=bool)
    insample[sample] = True
    got = {(int(a), int(b)) for a, b in pairs0[insample[pairs0[:, 0]] | insample[pairs0[:, 1]]]}
    gp = idx[o.pairs()]
    ref = {(int(a), int(b)) for a, b in gp[insample[gp[:, 0]] | insample[gp[:, 1]]]}
    assert got == ref and len(ref) > 0
    o.step(steps)
    xo, vo, wo, ao = o.state()
    Fo, Mo = o.forces()
    Fa, Ma = o.force_scales()
    ks = lut[sample]
    assert np.array_equal(ag[sample], ao[ks])
    if precision == "fp64":
        for a, b in ((xg, xo), (vg, vo), (wg, wo), (Fg, Fo), (Mg, Mo)):
            assert np.array_equal(a[sample], b[ks])
    else:
        m = masses(sub)[ks]
        ef = force_error(Fg[sample], Fo[ks], Fa[ks], m, wl.cfg["gravity"])
        em = torque_error(Mg[sample], Mo[ks], Ma[ks], m, wl.radius[sample].astype(float), wl.cfg["gravity"])
        print(f"{wl.name} n={wl.n} sampled mixed error after {steps} steps: force {ef:.3e} torque {em:.3e}")
        assert ef <= MIXED_TOL and em <= MIXED_TOL
        dt = wl.cfg["dt"]
        a_scale = float(np.max(Fa[ks] / m)) + 9.81
        assert np.abs(xg[sample] - xo[ks]).max() <= MIXED_TOL * a_scale * dt * dt * steps * steps
    assert Fa[ks].sum() > 0                 # the sample does have contacts


def test_full_size_silo_mixed_sampled():
    # 4.3M spheres, packed bed (every sphere touches its lattice neighbours)
    wl = workloads.silo(precision="mixed", spacing=0.995, jitter=0.002)
    sampled_parity(wl, "mixed", steps=4)


def test_full_size_silo_fp64_sampled():
    wl = workloads.silo(precision="fp64", spacing=0.995, jitter=0.002)
    sampled_parity(wl, "fp64", steps=3)


def test_full_size_drum_sampled():
    # 200k polydisperse spheres; FCC at 0.999 d_max: the largest neighbours touch.  FP64
    # from rest (bit-exact); mixed from random spins of ~1 rad/s, because from rest the
    # constant rolling model turns rounding noise into spins (test_model_properties.py)
    sampled_parity(workloads.drum(precision="fp64", spacing=0.999), "fp64", steps=4)
    sampled_parity(workloads.drum(precision="mixed", spacing=0.999, spin=1.0), "mixed", steps=4)


def test_mixed_pair_once_equals_both_sides_up_to_the_order_of_the_sums():
    """Evaluating each touching pair once (by the partner of smaller id, its reaction handed
    to the other) or from both sides applies the same law to the same pairs: the tangential
    overlaps after an evaluation are bit-identical, the pair sets and contact counts equal,
    and the force sums differ only by the order of FP32 additions."""
    wl = dense(n=3000, seed=41, speed=1.0)
    runs = {}
    for mode in ("once", "both"):
        wl.cfg["pair_eval"] = mode
        g, o = make_gpu(wl, "mixed"), make_oracle(wl)
        with_history(wl, g, o)
        runs[mode] = (g, g.forces(), g.history(), g.pairs(), g.stats())
    Fa, Ma = o.force_scales()
    m = masses(wl)
    gvec = wl.cfg["gravity"]
    (g1, (F1, M1), h1, p1, s1), (g2, (F2, M2), h2, p2, s2) = runs["once"], runs["both"]
    assert np.array_equal(p1, p2)
    assert np.array_equal(h1[0], h2[0]) and np.array_equal(h1[1], h2[1]) and np.array_equal(h1[2], h2[2])
    assert s1["n_touch"] == s2["n_touch"] > 1000 and s1["n_wall_touch"] == s2["n_wall_touch"]
    ef = force_error(F1, F2, Fa, m, gvec)
    em = torque_error(M1, M2, Ma, m, wl.radius.astype(float), gvec)
    print(f"once vs both: force {ef:.2e} torque {em:.2e}")
    assert ef <= 1e-6 and em <= 1e-6
    for g in (g1, g2):
        g.step(50)
    x1, v1, _, a1 = g1.state()
    x2, v2, _, a2 = g2.state()
    assert np.array_equal(a1, a2)
    assert np.abs(x1 - x2).max() < 1e-9
