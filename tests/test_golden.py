"""Pins against numbers the paper prints (fixtures in tests/golden/, each citing its table).

  integration_order.txt .... Table integration_order: the orders of convergence that the
                             paper's explicit-Euler and velocity-Verlet errors imply (about 1
                             and 2) match the orders of the oracle's integrators on a contact
                             oscillation (the paper's test problem itself is not specified)
  weak_scaling.txt ......... Table weak_scaling: the dam-break generator's depth rule gives
                             the printed box depth for every printed particle count
  contact_properties.txt ... Table contact_properties: with the paper's particle-wall
                             properties, the oracle's wall impacts rebound with the input
                             restitution at both ends of the printed speed range
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table(name):
    rows = []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def orders(errs):
    return [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]


def test_integrator_orders_match_the_papers_table():
    rows = table("integration_order.txt")
    dts = [float(r[0]) for r in rows]
    assert all(abs(dts[k] / dts[k + 1] - 2.0) < 1e-12 for k in range(2))   # halved each time
    paper = {1: orders([float(r[1]) for r in rows]), 0: orders([float(r[2]) for r in rows])}
    assert all(abs(o - 1.0) < 0.1 for o in paper[1]) and all(abs(o - 2.0) < 0.1 for o in paper[0])

    # the oracle on a sphere oscillating on its Hertz contact with a floor (e = 1)
    G = 9.81
    m = dict(young=1e7, poisson=0.3, restitution=1.0, mu_slide=0.3, mu_roll=0.0)
    R = float(np.float32(1.5e-3))
    estar = 1.0 / (2 * (1 - 0.3 ** 2) / 1e7)
    K = 4.0 / 3.0 * estar * math.sqrt(R)
    d_eq = (2500.0 * 4.0 / 3.0 * math.pi * R ** 3 * G / K) ** (2.0 / 3.0)
    T = 2e-4

    def z_at(dt, integ):
        c = dict(density=2500.0, particle=m, wall=m, gravity=(0.0, 0.0, -G), dt=dt, neighbor_factor=1.3,
                 skin=0.0, rebuild_every=0, rolling_model=1, integrator=integ,
                 domain_lo=(-0.1, -0.1, -0.1), domain_hi=(0.1, 0.1, 0.1))
        s = oracle.OracleSim(c, np.array([[0.0, 0.0, R - 0.5 * d_eq]]), np.zeros((1, 3)), np.zeros((1, 3)),
                             np.array([R], np.float32), [workloads.plane((0, 0, 0), (0, 0, 1))])
        s.step(int(round(T / dt)))
        x, _, _, _ = s.state()
        return x[0, 2]

    for integ in (1, 0):
        ref = z_at(2e-6 / 128, integ)
        ours = orders([abs(z_at(dt, integ) - ref) for dt in (2e-6, 1e-6, 5e-7)])
        assert all(abs(a - b) < 0.15 for a, b in zip(ours, paper[integ])), (integ, ours, paper[integ])


def test_dam_break_depth_follows_the_weak_scaling_table():
    for n_c, per_core, z, n_p in table("weak_scaling.txt"):
        assert int(n_c) * int(per_core) == int(n_p)
        assert abs(workloads.dam_break_depth(int(n_p)) - float(z)) < 1e-12, (n_p, z)


@pytest.mark.parametrize("e", [0.5, 0.9])
@pytest.mark.parametrize("which_speed", ["impact_speed_min", "impact_speed_max"])
def test_wall_restitution_with_the_papers_contact_properties(e, which_speed):
    p = {r[0]: float(r[1]) for r in table("contact_properties.txt")}
    assert p["restitution_min"] <= e <= p["restitution_max"]
    v0 = p[which_speed]
    mat = dict(young=p["young"], poisson=p["poisson"], restitution=e, mu_slide=p["mu"], mu_roll=0.0)
    R = float(np.float32(0.5 * p["d_p"]))
    # Hertz contact time 3.21807 (m / (K sqrt(v)))^(2/5) for a sphere on a rigid-mass wall
    m = p["rho_p"] * 4.0 / 3.0 * math.pi * R ** 3
    K = 4.0 / 3.0 * (1.0 / (2 * (1 - p["poisson"] ** 2) / p["young"])) * math.sqrt(R)
    tc = 3.21807 * (m / (K * math.sqrt(v0))) ** 0.4
    dt = tc / 2000.0
    c = dict(density=p["rho_p"], particle=mat, wall=mat, gravity=(0.0, 0.0, 0.0), dt=dt, neighbor_factor=1.3,
             skin=0.0, rebuild_every=0, rolling_model=0, domain_lo=(-0.1, -0.1, -0.1), domain_hi=(0.1, 0.1, 0.1))
    s = oracle.OracleSim(c, np.array([[0.0, 0.0, R + 1e-3 * v0 * dt]]), np.array([[0.0, 0.0, -v0]]),
                         np.zeros((1, 3)), np.array([R], np.float32), [workloads.plane((0, 0, 0), (0, 0, 1))])
    s.step(int(1.5 * tc / dt) + 10)
    _, v, _, _ = s.state()
    assert abs(v[0, 2] / v0 - e) < 5e-4, (e, v0, v[0, 2] / v0)
