"""Invariants of the method checked on the CUDA path directly, in both precisions (the same
facts pin the oracle): a removed sphere exerts no force on a partner still in its list;
pair forces conserve momentum; pair torques change the total angular momentum only by the
overlap's lever; without dissipation the energy is conserved to second order in dt."""
import math

import numpy as np
import pytest

import workloads
from gpu_helpers import make_gpu

pytestmark = pytest.mark.gpu

G = 9.81


def material():
    return dict(young=1e7, poisson=0.3, restitution=0.9, mu_slide=0.3, mu_roll=0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_a_removed_sphere_exerts_no_force(precision):
    # A leaves at the first drift (z_sink just below it); B starts 0.1 d above contact with
    # A, in A's fine-search list, and falls through the place where A was frozen before any
    # new search: its fall must stay the exact free fall.
    R = float(np.float32(1.5e-3))
    d = 2 * R
    dt = 1e-5
    cfg = dict(density=2500.0, particle=material(), wall=material(), gravity=(0.0, 0.0, -G), dt=dt,
               neighbor_factor=1.3, skin=0.5 * d, rebuild_every=0, rolling_model=1, z_sink=-1e-12,
               domain_lo=(-0.02, -0.02, -0.02), domain_hi=(0.02, 0.02, 0.02))
    x = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.1 * d]])
    wl = workloads.Workload("pair", cfg, [], x, np.zeros((2, 3)), np.zeros((2, 3)),
                            np.array([R, R], np.float32))
    g = make_gpu(wl, precision)
    steps = 1000
    g.step(steps)
    xs, _, _, act = g.state()
    st = g.stats()
    g.close()
    t = steps * dt
    assert act.tolist() == [0, 1]
    assert xs[1, 2] < xs[0, 2] + 0.95 * d
    # FP64: exact up to rounding; mixed: gravity enters as an FP32 constant
    tol = 1e-12 if precision == "fp64" else 1e-10
    assert abs(xs[1, 2] - (1.1 * d - 0.5 * G * t * t)) < tol
    assert st["rebuilds"] == 1


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_angular_momentum_changes_only_by_the_overlap_lever(precision):
    wl = workloads.lattice(n=343, seed=7, walls=False, gravity=(0, 0, 0), speed=0.2)
    wl.cfg["domain_lo"] = (-0.01, -0.01, -0.01)
    wl.cfg["domain_hi"] = (0.04, 0.04, 0.04)
    for m_ in (wl.cfg["particle"], wl.cfg["wall"]):
        m_["young"] = 1e8
    wl.cfg["dt"] = 4e-6
    R = wl.radius.astype(np.float64)
    m = 2500.0 * 4.0 / 3.0 * math.pi * R ** 3
    inertia = 0.4 * m * R ** 2

    def ang(x, v, w):
        return (m[:, None] * np.cross(x, v)).sum(0) + (inertia[:, None] * w).sum(0)

    g = make_gpu(wl, precision)
    g.step(1)
    assert g.stats()["n_touch"] > 100
    g.step(749)
    x, v, w, _ = g.state()
    g.close()
    spin_change = np.linalg.norm(inertia[:, None] * (w - wl.w), axis=1).sum()
    ratio = np.linalg.norm(ang(x, v, w) - ang(wl.x, wl.v, wl.w)) / spin_change
    print(f"{precision}: |dL| / sum |I dw| = {ratio:.2e}")
    assert ratio < 3e-3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_momentum_conserved_by_pair_forces(precision):
    # both sides of a pair compute exactly opposite forces in either precision; the mixed
    # path then rounds each particle's force sum to FP32 before the FP64 update
    wl = workloads.lattice(n=343, seed=7, walls=False, gravity=(0, 0, 0), speed=0.2)
    wl.cfg["domain_lo"] = (-0.01, -0.01, -0.01)
    wl.cfg["domain_hi"] = (0.04, 0.04, 0.04)
    m = 2500.0 * 4.0 / 3.0 * math.pi * wl.radius.astype(np.float64) ** 3
    p0 = (m[:, None] * wl.v).sum(0)
    scale = (m[:, None] * np.abs(wl.v)).sum()
    g = make_gpu(wl, precision)
    g.step(1)
    assert g.stats()["n_touch"] > 300
    g.step(299)
    _, v, _, _ = g.state()
    g.close()
    drift = np.abs((m[:, None] * v).sum(0) - p0).max() / scale
    print(f"{precision}: momentum drift {drift:.2e}")
    assert drift < (1e-13 if precision == "fp64" else 1e-5)


def hertz_energy(cfg, x, v, w, R, walls):
    """Kinetic + potential energy with the Hertz elastic energy 2/5 k_n delta^2.5 of every
    particle-particle and particle-plane overlap."""
    def estar(a, b):
        return 1.0 / ((1 - a["poisson"] ** 2) / a["young"] + (1 - b["poisson"] ** 2) / b["young"])
    m = cfg["density"] * 4.0 / 3.0 * math.pi * R ** 3
    g = np.array(cfg["gravity"])
    E = 0.5 * (m[:, None] * v * v).sum() + 0.5 * (0.4 * m[:, None] * R[:, None] ** 2 * w * w).sum()
    E -= (m * (x @ g)).sum()
    iu = np.triu_indices(len(R), 1)
    dist = np.sqrt(((x[None, :, :] - x[:, None, :]) ** 2).sum(-1))[iu]
    ov = (R[:, None] + R[None, :])[iu] - dist
    Re = (R[:, None] * R[None, :] / (R[:, None] + R[None, :]))[iu]
    sel = ov > 0
    E += (0.4 * 4.0 / 3.0 * estar(cfg["particle"], cfg["particle"]) * np.sqrt(Re[sel]) * ov[sel] ** 2.5).sum()
    kw = 4.0 / 3.0 * estar(cfg["particle"], cfg["wall"]) * np.sqrt(R)
    for wall in walls:
        nrm = np.array(wall["normal"]) / np.linalg.norm(wall["normal"])
        o = R - (x - np.array(wall["point"])) @ nrm
        sel = o > 0
        E += (0.4 * kw[sel] * o[sel] ** 2.5).sum()
    return E


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_conserved_without_dissipation_to_second_order(precision):
    drifts = []
    for dt in (4e-6, 2e-6):
        wl = workloads.lattice(n=216, seed=11, spacing=1.05, speed=0.3, spin=0.0)
        for m_ in (wl.cfg["particle"], wl.cfg["wall"]):
            m_.update(restitution=1.0, mu_slide=0.0, mu_roll=0.0)
        wl.cfg["dt"] = dt
        R = wl.radius.astype(np.float64)
        E0 = hertz_energy(wl.cfg, wl.x, wl.v, wl.w, R, wl.walls)
        ke0 = 0.5 * (2500.0 * 4.0 / 3.0 * math.pi * R[:, None] ** 3 * wl.v ** 2).sum()
        g = make_gpu(wl, precision)
        worst = 0.0
        for _ in range(10):
            g.step(int(round(0.004 / dt / 10)))
            x, v, w, _ = g.state()
            worst = max(worst, abs(hertz_energy(wl.cfg, x, v, w, R, wl.walls) - E0) / ke0)
        assert g.stats()["n_touch"] > 0
        g.close()
        drifts.append(worst)
    print(f"{precision}: energy drift {drifts[0]:.2e} (dt 4e-6), {drifts[1]:.2e} (dt 2e-6)")
    assert drifts[0] < 1e-3
    assert drifts[1] < drifts[0] / 2.5
