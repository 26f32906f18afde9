"""Pins of the oracle's variants of the method (the paper's other options, Sec. 2.1-2.2):
the linear contact model (Eqs. linearkn, linearetan), the viscous rolling resistance
(Table rolling_torque), the explicit Euler integrator (Eq. integ_EE) and walls whose
geometry translates (Sec. 3.6).  Each against a closed form:

  linear stiffness ..... k_n is the spring that gives Hertz's maximum overlap at impact speed
                         V; a linear spring's contact time pi sqrt(m_e / k_n) is independent
                         of the impact speed and its maximum overlap scales with it
  linear restitution ... eta_n of Eq. linearetan gives back the input e (spring-dashpot)
  viscous rolling ...... a rolling sphere decays as exp(-5/7 mu_r g t)
  explicit Euler ....... free fall follows the exact discrete recursion; order 1 (Verlet: 2)
  translating wall ..... a plate moving at U hits a resting sphere when the gap closes and
                         sends it off at 2 U (elastic, frictionless, infinitely heavy wall)
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from test_oracle_pins import FLOOR, G, cfg, crossing_times, estar, f32, mass, mat, sim1


def linear_two_sphere(e, v_rel, V, R=float(np.float32(1e-3)), rho=7850.0, young=2e11, nu=0.3, steps=4000):
    """Two equal spheres head-on with the linear model; returns distances, velocities,
    dt, the linear contact time pi sqrt(m_e / k_n) and Hertz's maximum overlap at V."""
    m = mat(young=young, poisson=nu, restitution=e, mu_slide=0.0)
    me = mass(R, rho) / 2.0
    Re = R / 2.0
    Ye = estar(m, m)
    dmax_hertz = (15.0 * me * V ** 2 / (16.0 * math.sqrt(Re) * Ye)) ** 0.4
    kn = me * V ** 2 / dmax_hertz ** 2            # the spring with Hertz's overlap at V
    tc = math.pi * math.sqrt(me / kn)
    dt = tc / steps
    gap = 0.5 * v_rel * dt * 10
    x = np.array([[-R - gap, 0.0, 0.0], [R + gap, 0.0, 0.0]])
    v = np.array([[0.5 * v_rel, 0, 0], [-0.5 * v_rel, 0, 0]])
    c = cfg(particle=m, wall=m, density=rho, gravity=(0, 0, 0), dt=dt, contact_model=1, linear_velocity=V,
            domain_lo=(-0.01, -0.01, -0.01), domain_hi=(0.01, 0.01, 0.01))
    s = oracle.OracleSim(c, x, v, np.zeros((2, 3)), np.array([R, R], np.float32))
    dist, vel = [], []
    for _ in range(int(2.5 * steps)):
        s.step(1)
        xx, vv, _, _ = s.state()
        dist.append(np.linalg.norm(xx[1] - xx[0]))
        vel.append(vv.copy())
    return np.array(dist), np.array(vel), dt, tc, dmax_hertz


def test_linear_stiffness_gives_hertz_overlap_at_the_characteristic_speed():
    V = 0.8
    R = f32(1e-3)
    dist, vel, dt, tc, dmax_h = linear_two_sphere(1.0, V, V)
    assert abs((2 * R - dist.min()) - dmax_h) / dmax_h < 1e-4
    t = crossing_times(dist, 2 * R, dt)
    assert len(t) == 2 and abs((t[1] - t[0]) - tc) / tc < 1e-3
    # a linear spring: same contact time, overlap proportional to the impact speed
    for f in (0.5, 2.0):
        d2, _, dt2, tc2, _ = linear_two_sphere(1.0, f * V, V)
        t2 = crossing_times(d2, 2 * R, dt2)
        assert abs((t2[1] - t2[0]) - tc) / tc < 1e-3
        assert abs((2 * R - d2.min()) - f * dmax_h) / (f * dmax_h) < 2e-4


@pytest.mark.parametrize("e", [0.5, 0.8, 0.95])
def test_linear_damping_recovers_the_input_restitution(e):
    V = 1.0
    dist, vel, *_ = linear_two_sphere(e, 0.6, V, steps=6000)
    e_rec = (vel[-1][1, 0] - vel[-1][0, 0]) / 0.6
    assert abs(e_rec - e) < 3e-4


def test_viscous_rolling_decays_exponentially():
    mu_r = 2.0      # s/m: the viscous model multiplies the constant one by |V_omega|
    wm = mat(restitution=0.5, mu_slide=0.8, mu_roll=mu_r)
    R = f32(1.5e-3)
    c = cfg(wall=wm, particle=mat(restitution=0.5), dt=2e-6, rolling_model=2)
    K = 4.0 / 3.0 * estar(c["particle"], wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    v0 = 0.2
    s = sim1(c, (0, 0, R - d_eq), v=(v0, 0, 0), w=(0, v0 / R, 0), R=R, walls=FLOOR)
    s.step(2000)
    _, va, _, _ = s.state()
    s.step(20000)
    _, vb, _, _ = s.state()
    rate = math.log(va[0, 0] / vb[0, 0]) / (20000 * 2e-6)
    expect = 5.0 / 7.0 * mu_r * G
    assert abs(rate - expect) / expect < 1e-2


def test_explicit_euler_free_fall_follows_the_discrete_recursion():
    dt = 1e-4
    c = cfg(dt=dt, integrator=1)
    z0, v0 = 0.05, 0.3
    s = sim1(c, (0, 0, z0), v=(0, 0, v0))
    for n in (1, 7, 100):
        s.step(n if n == 1 else n - (1 if n == 7 else 7))
        x, v, _, _ = s.state()
        assert abs(v[0, 2] - (v0 - G * n * dt)) <= 1e-12
        assert abs(x[0, 2] - (z0 + v0 * n * dt - G * dt * dt * n * (n - 1) / 2)) <= 1e-12


def test_explicit_euler_is_first_order_where_verlet_is_second():
    pm = mat(restitution=1.0)
    R = f32(1.5e-3)
    K = 4.0 / 3.0 * estar(pm, pm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    T = 2e-4

    def z_at(dt, integ):
        c = cfg(particle=pm, wall=pm, dt=dt, integrator=integ)
        s = sim1(c, (0, 0, R - 0.5 * d_eq), R=R, walls=FLOOR)
        s.step(int(round(T / dt)))
        x, _, _, _ = s.state()
        return x[0, 2]

    for integ, order in ((1, 1.0), (0, 2.0)):
        ref = z_at(2e-6 / 128, integ)
        errs = [abs(z_at(dt, integ) - ref) for dt in (2e-6, 1e-6, 5e-7)]
        orders = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
        assert all(abs(o - order) < 0.15 for o in orders), (integ, orders)


def test_translating_wall_hits_and_throws_a_resting_sphere():
    U = 0.2
    R = f32(1.5e-3)
    pm = mat(restitution=1.0, mu_slide=0.0)
    dt = 1e-6
    c = cfg(particle=pm, wall=pm, gravity=(0, 0, 0), dt=dt, rolling_model=0)
    gap = 2e-4
    plate = [workloads.plane((0, 0, -gap), (0, 0, 1), velocity=(0, 0, U), translates=1)]
    s = sim1(c, (0, 0, R), R=R, walls=plate)
    t_hit = gap / U                                  # the plate reaches the sphere's surface
    s.step(int(t_hit / dt) - 2)
    _, v, _, _ = s.state()
    assert v[0, 2] == 0.0
    s.step(4)
    _, v, _, _ = s.state()
    assert v[0, 2] > 0.0
    s.step(4000)
    _, v, _, _ = s.state()
    assert abs(v[0, 2] - 2 * U) / (2 * U) < 1e-3


def test_linear_tangential_stiffness_equals_normal():
    # On a floor the tangential mode obeys u'' = -(7/2) k_t / m u (I = 2/5 m R^2); the linear
    # model takes k_t = k_n, the Hertz-equivalent spring at the characteristic speed V.
    V = 0.5
    pm = mat(restitution=0.9)
    wm = mat(young=4e7, poisson=0.2, restitution=1.0, mu_slide=10.0, mu_roll=0.0)
    R = f32(1.5e-3)
    m = mass(R)
    Ye = estar(pm, wm)
    kn = m * V ** 2 / (15.0 * m * V ** 2 / (16.0 * math.sqrt(R) * Ye)) ** 0.8
    d_eq = m * G / kn
    dt = 2e-7
    c = cfg(particle=pm, wall=wm, dt=dt, rolling_model=0, contact_model=1, linear_velocity=V)
    s = sim1(c, (0, 0, R - d_eq), v=(1e-4, 0, 0), R=R, walls=FLOOR)
    ut = []
    for _ in range(40000):
        s.step(1)
        _, _, dtw = s.history()
        ut.append(dtw[0, 0, 0])
    T = 2 * math.pi / math.sqrt(3.5 * kn / m)
    z = crossing_times(np.array(ut), 0.0, dt)
    assert len(z) > 6
    T_meas = (z[-1] - z[1]) / ((len(z) - 2) / 2.0)
    assert abs(T_meas - T) / T < 1e-4


def test_explicit_euler_sliding_then_rolling_five_sevenths():
    # The rotational update of the Euler step: a sphere sliding on a floor ends rolling at
    # 5/7 of its initial speed (first-order scheme: 2e-3 at this step size, as Verlet)
    mu = 0.3
    wm = mat(restitution=0.5, mu_slide=mu, mu_roll=0.0)
    R = f32(1.5e-3)
    c = cfg(wall=wm, particle=mat(restitution=0.5), dt=2e-6, rolling_model=0, integrator=1)
    K = 4.0 / 3.0 * estar(c["particle"], wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    v0 = 0.2
    s = sim1(c, (0, 0, R - d_eq), v=(v0, 0, 0), R=R, walls=FLOOR)
    s.step(int(3.0 * 2 * v0 / (7 * mu * G) / 2e-6))
    _, v, w, _ = s.state()
    assert abs(v[0, 0] - 5.0 / 7.0 * v0) / v0 < 2e-3
    assert abs(w[0, 1] - v[0, 0] / R) / (v[0, 0] / R) < 2e-3


def test_explicit_euler_removes_a_sphere_below_z_sink():
    # Euler free fall z_n = z0 - g dt^2 n (n - 1) / 2 (exact recursion): the sphere leaves at
    # the first step whose height is below z_sink, placed halfway between two steps
    dt, z0 = 1e-4, 0.05
    n_star = 60

    def z(n):
        return z0 - G * dt * dt * n * (n - 1) / 2

    c = cfg(dt=dt, integrator=1, z_sink=0.5 * (z(n_star - 1) + z(n_star)))
    s = sim1(c, (0.0, 0.0, z0))
    s.step(n_star - 1)
    assert s.state()[3][0] == 1
    s.step(1)
    x, _, _, act = s.state()
    assert act[0] == 0 and abs(x[0, 2] - z(n_star)) < 1e-12
