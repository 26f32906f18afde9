"""The CUDA path against closed forms of contact mechanics, in both precisions: the mixed
path's FP32 contact law, integrated over whole contacts, must reproduce what the method
fixes as well as the FP64 path does (the same facts pin the oracle)."""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

G = 9.81


def mat(**kw):
    m = dict(young=1e7, poisson=0.3, restitution=0.9, mu_slide=0.3, mu_roll=0.0)
    m.update(kw)
    return m


def cfg(**kw):
    c = dict(density=2500.0, particle=mat(), wall=mat(), gravity=(0.0, 0.0, -G), dt=1e-5,
             neighbor_factor=1.3, skin=0.0, rebuild_every=0, rolling_model=1,
             domain_lo=(-0.1, -0.1, -0.1), domain_hi=(0.1, 0.1, 0.1))
    c.update(kw)
    return c


def f32(r):
    return float(np.float32(r))


def mass(R, rho=2500.0):
    return rho * 4.0 / 3.0 * math.pi * R ** 3


def estar(m1, m2):
    """Hertz contact modulus 1/E* = (1-nu1^2)/E1 + (1-nu2^2)/E2."""
    return 1.0 / ((1 - m1["poisson"] ** 2) / m1["young"] + (1 - m2["poisson"] ** 2) / m2["young"])


FLOOR = [workloads.plane((0, 0, 0), (0, 0, 1))]


def run(precision, c, x, v, R, walls, steps):
    from paper_2106_09576_gb300 import DEM
    x = np.array(x, float).reshape(-1, 3)
    n = len(x)
    g = DEM(c, x, np.array(v, float).reshape(n, 3), np.zeros((n, 3)), np.full(n, R, np.float32), walls,
            precision=precision)
    g.step(steps)
    out = g.state()
    g.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_overlap_on_plane_matches_hertz(precision):
    pm = mat(restitution=0.3)
    wm = mat(young=5e7, poisson=0.25, restitution=0.3)
    R = f32(1.5e-3)
    x, v, _, _ = run(precision, cfg(particle=pm, wall=wm, dt=2e-6), (0, 0, R), (0, 0, 0), R, FLOOR, 60000)
    K = 4.0 / 3.0 * estar(pm, wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    err = abs((R - x[0, 2]) - d_eq) / d_eq
    print(f"{precision}: static overlap relative error {err:.2e}")
    assert abs(v[0, 2]) < 1e-9
    assert err < (1e-6 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_static_overlap_in_a_horizontal_cylinder_matches_hertz(precision):
    # the sphere rests at the bottom of a drum (axis along y, 8 cm radius, off the origin):
    # the wall model takes the sphere's own radius as the contact radius, so the overlap is
    # the plane's, 8e-7 m against a distance from the axis of 8e-2 m -- an FP32 radial
    # distance alone would be off by ~5e-9 m, 0.6 % of it
    pm = mat(restitution=0.3)
    wm = mat(young=5e7, poisson=0.25, restitution=0.3)
    R = f32(1.5e-3)
    Rc, x0 = 0.08, 0.013
    drum = [workloads.cylinder((x0, 0.0, Rc), (0, 1, 0), Rc)]
    c = cfg(particle=pm, wall=wm, dt=2e-6, domain_lo=(-0.1, -0.1, -0.01), domain_hi=(0.1, 0.1, 0.19))
    x, v, _, _ = run(precision, c, (x0, 0, R), (0, 0, 0), R, drum, 60000)
    K = 4.0 / 3.0 * estar(pm, wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    rho = math.hypot(x[0, 0] - x0, x[0, 2] - Rc)
    err = abs((rho + R - Rc) - d_eq) / d_eq
    print(f"{precision}: static overlap in the cylinder, relative error {err:.2e}")
    assert abs(v[0, 2]) < 1e-9 and abs(x[0, 0] - x0) < 1e-9
    assert err < (1e-6 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("v_rel", [0.1, 2.0])
def test_restitution_recovers_input_coefficient(precision, v_rel):
    e = 0.7
    R = f32(1e-3)
    rho = 7850.0
    m = mat(young=2e11, poisson=0.3, restitution=e, mu_slide=0.0)
    me = mass(R, rho) / 2.0
    K = 4.0 / 3.0 * estar(m, m) * math.sqrt(R / 2.0)
    dmax = (5.0 * me * v_rel ** 2 / (4.0 * K)) ** 0.4
    tc = 2.94328 * dmax / v_rel
    dt = tc / 4000
    gap = 0.5 * v_rel * dt * 10
    c = cfg(particle=m, wall=m, density=rho, gravity=(0, 0, 0), dt=dt,
            domain_lo=(-0.01, -0.01, -0.01), domain_hi=(0.01, 0.01, 0.01))
    _, v, _, _ = run(precision, c, [[-R - gap, 0, 0], [R + gap, 0, 0]],
                     [[0.5 * v_rel, 0, 0], [-0.5 * v_rel, 0, 0]], R, [], 12000)
    e_rec = (v[1, 0] - v[0, 0]) / v_rel
    print(f"{precision}: v_rel {v_rel} restitution {e_rec:.6f}")
    assert abs(e_rec - e) < 2e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sliding_then_rolling_five_sevenths(precision):
    mu = 0.3
    wm = mat(restitution=0.5, mu_slide=mu, mu_roll=0.0)
    R = f32(1.5e-3)
    c = cfg(wall=wm, particle=mat(restitution=0.5), dt=2e-6, rolling_model=0)
    K = 4.0 / 3.0 * estar(c["particle"], wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    v0 = 0.2
    t_star = 2 * v0 / (7 * mu * G)
    steps = int(0.5 * t_star / 2e-6) + int(2.5 * t_star / 2e-6)
    _, v, w, _ = run(precision, c, (0, 0, R - d_eq), (v0, 0, 0), R, FLOOR, steps)
    print(f"{precision}: v / v0 = {v[0, 0] / v0:.6f} (5/7 = {5 / 7:.6f})")
    assert abs(v[0, 0] - 5.0 / 7.0 * v0) / v0 < 2e-3
    assert abs(w[0, 1] - v[0, 0] / R) / (v[0, 0] / R) < 2e-3       # rolls without slip
