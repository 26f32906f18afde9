"""The synthetic inputs follow the recipes they state: counts, radii, geometry, seeding, no
initial overlap where a recipe promises none, and touching neighbours where it promises
them (the packed silo of the benchmark)."""
import math

import numpy as np
import pytest

import bench
import workloads

cKDTree = pytest.importorskip("scipy.spatial").cKDTree


def overlapping_pairs(x, radius):
    """Number of overlapping pairs and the largest overlap."""
    r = radius.astype(np.float64)
    p = cKDTree(x).query_pairs(2.0 * float(r.max()), output_type="ndarray")
    if len(p) == 0:
        return 0, 0.0
    ov = r[p[:, 0]] + r[p[:, 1]] - np.linalg.norm(x[p[:, 0]] - x[p[:, 1]], axis=1)
    return int((ov > 0).sum()), float(max(ov.max(), 0.0))


# FCC sites 1.02 d_k apart, each moved by up to 0.01 d_k per coordinate: nearest neighbours
# lie along face diagonals, so two centres approach by at most 0.02 sqrt(2) d_k and spheres
# of diameter d_k overlap by at most (1 - 1.02 + 0.02 sqrt(2)) d_k
FCC_MAX_OVERLAP = 1.0 - 1.02 + 0.02 * math.sqrt(2.0)


def test_generators_are_seeded_and_repeatable():
    for make in (lambda s: workloads.drum(n=3000, seed=s), lambda s: workloads.lattice(n=500, seed=s),
                 lambda s: workloads.dam_break(n=3000, seed=s, depth=0.01)):
        a, b, c = make(5), make(5), make(6)
        for f in ("x", "v", "w", "radius"):
            assert np.array_equal(getattr(a, f), getattr(b, f))
        assert not np.array_equal(a.x, c.x)


def test_drum_recipe():
    wl = workloads.drum()
    R, L = wl.cfg["drum_radius"], wl.cfg["drum_length"]
    r = wl.radius.astype(np.float64)
    assert wl.n == 200_000 and wl.radius.dtype == np.float32
    assert r.min() >= np.float32(1.5e-3) and r.max() <= np.float32(2.5e-3)
    # the paper's aspect L/R = 0.1/0.12, scaled so that the spheres half fill it at phi = 0.6
    assert L / R == pytest.approx(0.1 / 0.12, rel=1e-12)
    assert R == pytest.approx(0.2085, abs=5e-4) and L == pytest.approx(0.1738, abs=5e-4)
    solid = float((4.0 / 3.0 * math.pi * r ** 3).sum())
    assert 0.27 < solid / (math.pi * R * R * L) <= 0.3 + 1e-12
    # every sphere inside the drum, and at most grazing another at t = 0
    x = wl.x
    assert (np.hypot(x[:, 0], x[:, 2]) + r <= R).all()
    assert (x[:, 1] - r >= 0.0).all() and (x[:, 1] + r <= L).all()
    count, worst = overlapping_pairs(x, wl.radius)
    assert worst <= FCC_MAX_OVERLAP * 5e-3 and count < 10
    # filled from the bottom: the lowest lattice sites first
    assert np.median(x[:, 2]) < 0.0
    # a cylinder and two end caps, all turning at 1 rad/s about the +y axis
    assert [w["kind"] for w in wl.walls] == [1, 0, 0]
    for w in wl.walls:
        assert w["omega"] == 1.0 and tuple(w["rot_axis"]) == (0.0, 1.0, 0.0)
    assert wl.cfg["dt"] == 5e-6 and np.all(wl.v == 0.0)


def test_packed_silo_of_the_benchmark():
    wl, desc = bench.make_workload("silo")
    d = 5e-3
    assert desc == "silo-packed" and wl.n == 4_300_000
    assert np.all(wl.radius == np.float32(0.5 * d))
    x = wl.x
    # inside the R = 0.5 m cylinder and above the bottom
    assert (np.hypot(x[:, 0], x[:, 1]) + 0.5 * d <= 0.5).all() and (x[:, 2] - 0.5 * d >= 0.0).all()
    # every sampled sphere touches all its lattice (face) neighbours and no other sphere
    tree = cKDTree(x)
    rng = np.random.default_rng(0)
    sample = rng.choice(wl.n, 5000, replace=False)
    touching = []
    for i, nb in zip(sample, tree.query_ball_point(x[sample], r=1.2 * d)):
        nb = [j for j in nb if j != i]
        dist = np.linalg.norm(x[nb] - x[i], axis=1)
        assert (dist < d).all() and (dist > 0.98 * d).all()
        assert len(nb) <= 6
        touching.append(len(nb))
    assert 5.5 < np.mean(touching) <= 6.0
    # search with a 0.5 d skin; the plug over the orifice holds the bed
    assert wl.cfg["skin"] == pytest.approx(0.5 * d)
    kinds = [w["kind"] for w in wl.walls]
    assert kinds == [1, 2, 0]
    assert wl.walls[1]["inner_radius"] == 0.05 and wl.walls[2]["t_off"] > 1e6


def test_batched_drums_recipe():
    wl = workloads.batched_drums()
    inst = wl.cfg["instances"]
    assert len(inst) == 512 and wl.n == 2_690_805
    counts = np.array([I["n"] for I in inst])
    assert counts.min() >= 500 and counts.max() <= 20_000 and counts.sum() == wl.n
    # log-uniform counts: the median near the geometric mean of the range
    assert abs(math.log(np.median(counts)) - 0.5 * (math.log(500) + math.log(20_000))) < 0.3
    firsts = [I["first"] for I in inst]
    assert firsts == list(np.concatenate([[0], np.cumsum(counts)[:-1]]))
    r = wl.radius.astype(np.float64)
    assert r.min() >= np.float32(1e-3) and r.max() <= np.float32(3e-3)
    rc = 1.3 * 2.0 * 3e-3
    boxes = []
    for I in inst:
        lo, n = I["first"], I["n"]
        xi, ri = wl.x[lo:lo + n], r[lo:lo + n]
        cx, y0, cz = I["center"][0], I["y0"], I["center"][2]
        R, L = I["radius"], I["length"]
        assert L / R == pytest.approx(0.1 / 0.12, rel=1e-12)
        assert (np.hypot(xi[:, 0] - cx, xi[:, 2] - cz) + ri <= R).all()
        assert (xi[:, 1] - ri >= y0).all() and (xi[:, 1] + ri <= y0 + L).all()
        assert 0.5 <= I["omega"] <= 3.0
        assert 0.2 <= I["particle"]["mu_slide"] <= 0.6 and 0.7 <= I["particle"]["restitution"] <= 0.95
        boxes.append((cx - R, y0, cz - R, cx + R, y0 + L, cz + R))
    # the drums' boxes are at least one search radius apart: no cross-instance candidate
    b = np.array(boxes)
    for k in range(len(b)):
        gap = np.maximum(b[k, :3] - b[:, 3:], b[:, :3] - b[k, 3:]).max(axis=1)
        gap[k] = np.inf
        assert gap.min() >= rc - 1e-12
    count, worst = overlapping_pairs(wl.x, wl.radius)
    assert worst <= FCC_MAX_OVERLAP * 6e-3 and count < 1e-5 * wl.n


def test_dam_break_recipe():
    n = 20_000
    wl = workloads.dam_break(n=n, seed=3)
    d = 1e-3
    depth = workloads.dam_break_depth(n)
    assert wl.n == n and np.all(wl.radius == np.float32(0.5 * d))
    x = wl.x
    # behind the dam (x < 0.1 m) in a box of the weak-scaling depth
    assert (x[:, 0] + 0.5 * d <= 0.1).all() and (x[:, 0] - 0.5 * d >= 0.0).all()
    assert (x[:, 1] - 0.5 * d >= 0.0).all() and (x[:, 1] + 0.5 * d <= depth).all()
    assert (x[:, 2] - 0.5 * d >= 0.0).all()
    # cubic lattice 1.05 d apart, moved by up to 0.02 d per coordinate: no overlap
    assert overlapping_pairs(x, wl.radius) == (0, 0.0)
    dam = wl.walls[-1]
    assert dam["kind"] == 0 and dam["point"][0] == 0.1 and dam["t_off"] == 0.05
    assert wl.cfg["dt"] == 4e-6


def test_instance_workload_is_the_batch_member_alone():
    wl = workloads.batched_drums(n_instances=8, n_lo=500, n_hi=900)
    for k in (0, 5, 7):
        I = wl.cfg["instances"][k]
        one = workloads.instance_workload(wl, k)
        lo, n = I["first"], I["n"]
        assert one.n == n and np.array_equal(one.x, wl.x[lo:lo + n]) and np.array_equal(one.radius, wl.radius[lo:lo + n])
        assert one.walls == I["walls"] and one.cfg["particle"] == I["particle"] and one.cfg["wall"] == I["wall"]
        assert "instances" not in one.cfg and "n_instances" not in one.cfg
        # its own domain holds the whole drum and a search radius around it
        dlo, dhi = np.array(one.cfg["domain_lo"]), np.array(one.cfg["domain_hi"])
        assert (one.x - one.radius[:, None] >= dlo).all() and (one.x + one.radius[:, None] <= dhi).all()
        assert dhi[1] - dlo[1] >= I["length"] and dhi[0] - dlo[0] >= 2 * I["radius"]
