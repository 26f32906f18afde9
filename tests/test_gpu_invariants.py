"""Invariants of the method checked on the CUDA path directly, in both precisions (the same
facts pin the oracle): a removed sphere exerts no force on a partner still in its list,
and pair torques change the total angular momentum only by the overlap's lever."""
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
