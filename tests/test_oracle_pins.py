"""Pins of the CPU oracle against closed forms, textbook results and invariants.

Each test states a result fixed by mechanics or by the paper's own definitions (not a
retyped oracle formula), chosen so that a plausible slip in the oracle (a dropped term,
a sign, a lever arm, an inertia factor, a mixing rule) fails at least one of them:

  free fall ............ velocity Verlet is exact under constant acceleration (Sec. 2.2)
  static overlap ....... Hertz sphere-on-flat law F = 4/3 E* sqrt(R) d^1.5 (k_n, Y_e mixing)
  head-on impact ....... Hertz contact time 2.94328 d_max / v (k_n, m_e, R_e, normal sign)
  restitution .......... the damping law recovers the input e for any impact speed (eta_n, beta)
  tangential mode ...... Mindlin stiffness 8 G* a with the 7/2 rolling factor (k_t, G_e, lever, I)
  tangential damping ... decay of the same mode (eta_t)
  sliding -> rolling ... v -> 5/7 v0 at t = 2 v0 / (7 mu g) (Coulomb limit, torque sign)
  rolling resistance ... dv/dt = -5/7 mu_r g (constant rolling torque, Table rolling_torque)
  moving walls ......... 2/7 V on a translating plate; turntable spin-up; drum drag direction
  cylinder, annulus .... static overlap on a curved wall; rim contact geometry
  floating wall ........ support until t_off, free fall after
  Coulomb .............. |F_t| <= mu |F_n| always; sliding at 65 deg, sticking at 5 deg;
                         no jump of F_t at the stick-slip switch (Sec. 2.1)
  momentum, energy ..... pair forces are equal and opposite; e = 1, mu = 0 conserves energy;
                         angular momentum changes only by the overlap lever (torque signs on i and j)
  search cadence ....... thin skin, thick skin and a search every step give the same bits
  z_sink ............... a falling sphere leaves at the step free fall predicts and stays put;
                         a removed sphere exerts no force
  constant search ...... a search before the first step, then one every n steps (Sec. 3.1)
  spinning pairs ....... meshing spins do not slip and feel only rolling resistance (exact);
                         equal spins slide with tangential impulse mu x normal impulse
  error scales ......... per-particle |F| and |M| sums of a sliding sphere, every evaluation anew
  invariance ........... wall contacts under translation; spheres that never meet move as if
                         alone; a translating turntable carries a co-moving sphere
  floating wall ........ present for t_on <= t < t_off (exact times with dt = 2^-16)
  integrator order ..... 2 for a smooth conservative contact oscillation
  contact search ....... cell list == O(n^2) brute force (NumPy), including r = r_c +- 1 ulp
"""
import math

import numpy as np
import pytest
from scipy.special import gamma

import oracle
import workloads

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


def sim1(c, x, v=(0, 0, 0), w=(0, 0, 0), R=1.5e-3, walls=()):
    return oracle.OracleSim(c, np.array([x], float), np.array([v], float),
                            np.array([w], float), np.array([R], np.float32), walls)


def f32(r):
    """Radii are FP32 inputs; closed forms use the value the simulation sees."""
    return float(np.float32(r))


def mass(R, rho=2500.0):
    return rho * 4.0 / 3.0 * math.pi * R ** 3


def estar(m1, m2):
    """Hertz contact modulus 1/E* = (1-nu1^2)/E1 + (1-nu2^2)/E2."""
    return 1.0 / ((1 - m1["poisson"] ** 2) / m1["young"] + (1 - m2["poisson"] ** 2) / m2["young"])


def gstar(m1, m2):
    """Mindlin shear modulus 1/G* = (2-nu1)/G1 + (2-nu2)/G2, G = E / (2(1+nu))."""
    g1 = m1["young"] / (2 * (1 + m1["poisson"]))
    g2 = m2["young"] / (2 * (1 + m2["poisson"]))
    return 1.0 / ((2 - m1["poisson"]) / g1 + (2 - m2["poisson"]) / g2)


FLOOR = [workloads.plane((0, 0, 0), (0, 0, 1))]


def test_free_fall_is_exact():
    c = cfg(dt=1e-5)
    s = sim1(c, (0.01, 0.02, 0.05), v=(0.3, -0.2, 1.0), w=(1.0, 2.0, 3.0))
    s.step(2000)
    t = 2000 * 1e-5
    x, v, w, _ = s.state()
    ref_x = np.array([0.01 + 0.3 * t, 0.02 - 0.2 * t, 0.05 + 1.0 * t - 0.5 * G * t * t])
    ref_v = np.array([0.3, -0.2, 1.0 - G * t])
    # exact in exact arithmetic; rounding adds at most ~2 ulp per step (2000 steps)
    assert np.allclose(x[0], ref_x, rtol=1e-12, atol=0)
    assert np.allclose(v[0], ref_v, rtol=1e-12, atol=0)
    assert np.array_equal(w[0], [1.0, 2.0, 3.0])


def settle_on(walls, x0, R, c, steps):
    s = sim1(c, x0, R=R, walls=walls)
    s.step(steps)
    return s


def test_static_overlap_on_plane_matches_hertz():
    pm = mat(restitution=0.3)
    wm = mat(young=5e7, poisson=0.25, restitution=0.3)
    R = f32(1.5e-3)
    c = cfg(particle=pm, wall=wm, dt=2e-6)
    s = settle_on(FLOOR, (0, 0, R), R, c, 60000)
    x, v, _, _ = s.state()
    K = 4.0 / 3.0 * estar(pm, wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    assert abs(v[0, 2]) < 1e-9
    assert abs((R - x[0, 2]) - d_eq) / d_eq < 1e-6


def two_sphere(e, v_rel, R=float(np.float32(1e-3)), rho=7850.0, young=2e11, nu=0.3, mu=0.0, steps_per_tc=2000,
               b=0.0):
    """Two equal spheres approaching along x with relative speed v_rel and impact
    parameter b (offset along y). Returns time series of the centre distance and
    velocities, plus the Hertz contact-time estimate used to pick dt."""
    m = mat(young=young, poisson=nu, restitution=e, mu_slide=mu, mu_roll=0.0)
    me = mass(R, rho) / 2.0
    Re = R / 2.0
    K = 4.0 / 3.0 * estar(m, m) * math.sqrt(Re)
    dmax = (5.0 * me * v_rel ** 2 / (4.0 * K)) ** 0.4
    tc = 2.94328 * dmax / v_rel
    dt = tc / steps_per_tc
    gap = 0.5 * v_rel * dt * 10
    x = np.array([[-R - gap, 0.0, 0.0], [R + gap, b, 0.0]])
    v = np.array([[0.5 * v_rel, 0, 0], [-0.5 * v_rel, 0, 0]])
    c = cfg(particle=m, wall=m, density=rho, gravity=(0, 0, 0), dt=dt,
            domain_lo=(-0.01, -0.01, -0.01), domain_hi=(0.01, 0.01, 0.01))
    s = oracle.OracleSim(c, x, v, np.zeros((2, 3)), np.array([R, R], np.float32))
    dist, vel = [], []
    n = int(3 * steps_per_tc)
    for _ in range(n):
        s.step(1)
        xx, vv, _, _ = s.state()
        dist.append(np.linalg.norm(xx[1] - xx[0]))
        vel.append(vv.copy())
    return np.array(dist), np.array(vel), dt, tc, dmax, K, me


def crossing_times(series, level, dt):
    """Times (in units of the sampled steps) where the series crosses `level`, linear
    interpolation between samples."""
    out = []
    for k in range(1, len(series)):
        a, b = series[k - 1] - level, series[k] - level
        if a == 0.0:
            out.append((k - 1) * dt)
        elif a * b < 0.0:
            out.append((k - 1 + a / (a - b)) * dt)
    return out


def test_hertz_head_on_contact_time_and_depth():
    v_rel = 1.0
    dist, vel, dt, tc_est, dmax, K, me = two_sphere(1.0, v_rel)
    R = f32(1e-3)
    t = crossing_times(dist, 2 * R, dt)
    assert len(t) == 2
    # Hertz: t_c = 2 (d_max/v) int_0^1 (1-u^{5/2})^{-1/2} du, the integral = (2/5) B(2/5, 1/2)
    coef = 2.0 * 0.4 * gamma(0.4) * gamma(0.5) / gamma(0.9)
    tc = coef * dmax / v_rel
    assert abs((t[1] - t[0]) - tc) / tc < 1e-3
    assert abs((2 * R - dist.min()) - dmax) / dmax < 1e-4
    # elastic and frictionless: the spheres exchange velocities
    assert np.allclose(vel[-1][0], [-0.5 * v_rel, 0, 0], atol=1e-6 * v_rel)


@pytest.mark.parametrize("e", [0.5, 0.7, 0.9])
@pytest.mark.parametrize("v_rel", [0.1, 1.0, 2.0])
def test_restitution_recovers_input_coefficient(e, v_rel):
    # The normal damping eta_n = -2 sqrt(5/6) beta sqrt(S_n m_e) with beta(e) makes the
    # rebound speed ratio equal to e, independent of speed (Sec. 2.1).
    dist, vel, dt, *_ = two_sphere(e, v_rel, steps_per_tc=4000)
    rel_after = vel[-1][1, 0] - vel[-1][0, 0]
    e_rec = rel_after / v_rel
    assert abs(e_rec - e) < 2e-4


def test_restitution_on_wall():
    wm = mat(restitution=0.6, young=3e7, poisson=0.2)
    R = f32(1.5e-3)
    c = cfg(wall=wm, gravity=(0, 0, 0), dt=2e-7)
    s = sim1(c, (0, 0, R + 1e-6), v=(0, 0, -0.5), R=R, walls=FLOOR)
    s.step(60000)
    _, v, _, _ = s.state()
    assert abs(v[0, 2] / 0.5 - 0.6) < 2e-4


def contact_mode(e_wall, steps, dt=2e-7, mu=10.0, vx0=1e-4):
    """Sphere at its static Hertz overlap on a floor, kicked tangentially; returns the
    particle-wall tangential overlap (x component) per step and the model constants."""
    pm = mat(restitution=0.9)
    wm = mat(young=4e7, poisson=0.2, restitution=e_wall, mu_slide=mu, mu_roll=0.0)
    R = f32(1.5e-3)
    m = mass(R)
    K = 4.0 / 3.0 * estar(pm, wm) * math.sqrt(R)
    d_eq = (m * G / K) ** (2.0 / 3.0)
    c = cfg(particle=pm, wall=wm, dt=dt, rolling_model=0)
    s = sim1(c, (0, 0, R - d_eq), v=(vx0, 0, 0), R=R, walls=FLOOR)
    ut = []
    for _ in range(steps):
        s.step(1)
        _, _, dtw = s.history()
        ut.append(dtw[0, 0, 0])
    kt = 8.0 * gstar(pm, wm) * math.sqrt(R * d_eq)
    return np.array(ut), dt, m, kt, s


def test_tangential_stiffness_mindlin_with_rolling_coupling():
    # u'' = -k_t (1/m + R^2/I) u = -(7/2) k_t / m u for a sphere on a flat (I = 2/5 m R^2).
    ut, dt, m, kt, _ = contact_mode(1.0, 40000)
    T = 2 * math.pi / math.sqrt(3.5 * kt / m)
    z = crossing_times(ut, 0.0, dt)
    assert len(z) > 6
    T_meas = (z[-1] - z[1]) / ((len(z) - 2) / 2.0)
    assert abs(T_meas - T) / T < 1e-4


def test_tangential_damping_decay_rate():
    # Linear tangential mode with damping 7/2 eta_t / m: amplitude ~ exp(-7/4 eta_t t / m),
    # eta_t = -2 sqrt(5/6) beta sqrt(k_t m) (S_t = k_t for this model).
    e = 0.8
    ut, dt, m, kt, _ = contact_mode(e, 30000)
    beta = math.log(e) / math.sqrt(math.log(e) ** 2 + math.pi ** 2)
    eta_t = -2 * math.sqrt(5.0 / 6.0) * beta * math.sqrt(kt * m)
    gam = 3.5 * eta_t / (2 * m)
    # peaks of |u|
    a = np.abs(ut)
    peaks = [k for k in range(1, len(a) - 1) if a[k] >= a[k - 1] and a[k] > a[k + 1]]
    t = np.array(peaks) * dt
    amp = a[peaks]
    fit = np.polyfit(t[:6], np.log(amp[:6]), 1)
    assert abs(-fit[0] - gam) / gam < 2e-2


def test_sliding_then_rolling_five_sevenths():
    mu = 0.3
    wm = mat(restitution=0.5, mu_slide=mu, mu_roll=0.0)
    R = f32(1.5e-3)
    # the particle material's own friction differs: against a wall the wall's mu applies (R8)
    c = cfg(wall=wm, particle=mat(restitution=0.5, mu_slide=0.7), dt=2e-6, rolling_model=0)
    K = 4.0 / 3.0 * estar(c["particle"], wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    v0 = 0.2
    s = sim1(c, (0, 0, R - d_eq), v=(v0, 0, 0), R=R, walls=FLOOR)
    t_star = 2 * v0 / (7 * mu * G)
    n1 = int(0.5 * t_star / 2e-6)
    s.step(n1)
    _, v, w, _ = s.state()
    assert abs(v[0, 0] - (v0 - mu * G * n1 * 2e-6)) / v0 < 2e-3       # decelerating at mu g
    s.step(int(2.5 * t_star / 2e-6))
    _, v, w, _ = s.state()
    assert abs(v[0, 0] - 5.0 / 7.0 * v0) / v0 < 2e-3
    assert abs(w[0, 1] - v[0, 0] / R) / (v[0, 0] / R) < 2e-3        # rolls without slip


def test_rolling_resistance_deceleration():
    mu_r = 0.1
    wm = mat(restitution=0.5, mu_slide=0.8, mu_roll=mu_r)
    R = f32(1.5e-3)
    c = cfg(wall=wm, particle=mat(restitution=0.5), dt=2e-6, rolling_model=1)
    K = 4.0 / 3.0 * estar(c["particle"], wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    v0 = 0.2
    s = sim1(c, (0, 0, R - d_eq), v=(v0, 0, 0), w=(0, v0 / R, 0), R=R, walls=FLOOR)
    s.step(2000)
    _, va, _, _ = s.state()
    s.step(20000)
    _, vb, _, _ = s.state()
    decel = (va[0, 0] - vb[0, 0]) / (20000 * 2e-6)
    assert abs(decel - 5.0 / 7.0 * mu_r * G) / (5.0 / 7.0 * mu_r * G) < 1e-2


def test_translating_plate_drags_sphere_to_two_sevenths():
    V = 0.1
    wm = mat(restitution=0.5, mu_slide=0.4)
    R = f32(1.5e-3)
    c = cfg(wall=wm, particle=mat(restitution=0.5), dt=2e-6, rolling_model=0)
    K = 4.0 / 3.0 * estar(c["particle"], wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    plate = [workloads.plane((0, 0, 0), (0, 0, 1), velocity=(V, 0, 0))]
    s = sim1(c, (0, 0, R - d_eq), R=R, walls=plate)
    s.step(40000)
    _, v, _, _ = s.state()
    assert abs(v[0, 0] - 2.0 / 7.0 * V) / V < 2e-3


def test_turntable_spin_up_by_rolling_torque():
    Om = 5.0
    mu_r = 0.2
    wm = mat(restitution=0.5, mu_slide=0.5, mu_roll=mu_r)
    R = f32(1.5e-3)
    c = cfg(wall=wm, particle=mat(restitution=0.5), dt=2e-6, rolling_model=1)
    K = 4.0 / 3.0 * estar(c["particle"], wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    table = [workloads.plane((0, 0, 0), (0, 0, 1), omega=Om, rot_origin=(0, 0, 0),
                             rot_axis=(0, 0, 1))]
    s = sim1(c, (0, 0, R - d_eq), R=R, walls=table)
    s.step(100)
    _, _, wa, _ = s.state()
    s.step(400)                      # Omega is reached only after ~765 steps
    _, _, wb, _ = s.state()
    rate = (wb[0, 2] - wa[0, 2]) / (400 * 2e-6)
    assert abs(rate - 2.5 * mu_r * G / R) / (2.5 * mu_r * G / R) < 1e-2
    # off the axis the surface velocity Omega x r drags the sphere along +y at x > 0
    s2 = sim1(c, (0.01, 0, R - d_eq), R=R, walls=table)
    s2.step(200)
    _, v, _, _ = s2.state()
    assert v[0, 1] > 0 and abs(v[0, 0]) < 0.05 * v[0, 1]


def test_cylinder_static_overlap_and_drum_drag():
    pm = mat(restitution=0.3)
    wm = mat(young=2e7, poisson=0.35, restitution=0.3)
    R = f32(1.5e-3)
    Rc = 0.05
    c = cfg(particle=pm, wall=wm, dt=2e-6)
    drum = [workloads.cylinder((0, 0, 0), (0, 1, 0), Rc)]
    s = settle_on(drum, (0, 0, -Rc + R), R, c, 60000)
    x, v, _, _ = s.state()
    K = 4.0 / 3.0 * estar(pm, wm) * math.sqrt(R)     # wall of infinite radius (R_e = R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    overlap = R - (Rc - math.hypot(x[0, 0], x[0, 2]))
    assert abs(overlap - d_eq) / d_eq < 1e-6
    # rotating about +y, the bottom of the drum moves along Omega x (p - c) = -x
    rot = [workloads.cylinder((0, 0, 0), (0, 1, 0), Rc, omega=2.0, rot_origin=(0, 0, 0),
                              rot_axis=(0, 1, 0))]
    s2 = oracle.OracleSim(c, x, np.zeros((1, 3)), np.zeros((1, 3)), np.array([R], np.float32), rot)
    s2.step(200)
    _, v2, _, _ = s2.state()
    assert v2[0, 0] < 0


def test_annulus_face_and_rim_contact_geometry():
    pm = mat(restitution=1.0)
    wm = mat(restitution=1.0, young=3e7)
    R = f32(2.5e-3)
    ring = [workloads.annulus((0, 0, 0), (0, 0, 1), 0.5, 0.004)]
    c = cfg(particle=pm, wall=wm, gravity=(0, 0, 0))
    K = 4.0 / 3.0 * estar(pm, wm) * math.sqrt(R)
    # face: centre 0.02 m from the axis, 2.4 mm above the plate
    s = sim1(c, (0.02, 0.0, 2.4e-3), R=R, walls=ring)
    F, _ = s.forces()
    assert np.allclose(F[0], [0, 0, K * (R - 2.4e-3) ** 1.5], rtol=1e-9, atol=1e-18)
    # rim: centre above the hole; nearest ring point found by sampling the rim circle
    xc = np.array([0.0025, 0.001, 1.5e-3])
    s = sim1(c, xc, R=R, walls=ring)
    F, _ = s.forces()
    from scipy.optimize import minimize_scalar

    def rim_pt(p):
        return np.array([0.004 * math.cos(p), 0.004 * math.sin(p), 0.0])

    phi = np.linspace(0, 2 * np.pi, 20001)
    k = int(np.argmin([np.linalg.norm(rim_pt(p) - xc) for p in phi]))
    best = minimize_scalar(lambda p: np.linalg.norm(rim_pt(p) - xc), method="bounded",
                           bounds=(phi[k] - 1e-3, phi[k] + 1e-3), options=dict(xatol=1e-13))
    p_near = rim_pt(best.x)
    dmin = np.linalg.norm(p_near - xc)
    delta = R - dmin
    direction = (xc - p_near) / dmin
    assert np.allclose(F[0], K * delta ** 1.5 * direction, rtol=1e-6, atol=1e-9 * K * delta ** 1.5)


def test_floating_wall_holds_until_t_off():
    R = f32(1.5e-3)
    t_off = 0.01
    c = cfg(particle=mat(restitution=0.3), wall=mat(restitution=0.3), dt=1e-5)
    plug = [workloads.plane((0, 0, 0), (0, 0, 1), t_off=t_off)]
    s = sim1(c, (0, 0, R), R=R, walls=plug)
    s.step(999)            # t = 9.99 ms: still supported
    x1, v1, _, _ = s.state()
    assert x1[0, 2] > R - 1e-4 and abs(v1[0, 2]) < 1e-3
    s.step(1001)           # 10 ms after the wall disappears
    x2, v2, _, _ = s.state()
    assert abs(v2[0, 2] - (v1[0, 2] - G * 1001 * 1e-5)) < 2e-3 * G * 1001 * 1e-5


def oblique_impact(angle):
    m = mat(young=2e11, poisson=0.3, restitution=0.7, mu_slide=0.3, mu_roll=0.0)
    R = f32(1e-3)
    V = 1.0
    a = math.radians(angle)
    me = mass(R, 7850.0)
    K = 4.0 / 3.0 * estar(m, m) * math.sqrt(R)
    dmax = (5 * me * V ** 2 / (4 * K)) ** 0.4
    dt = 2.94328 * dmax / (V * math.cos(a)) / 2000
    c = cfg(particle=m, wall=m, density=7850.0, gravity=(0, 0, 0), dt=dt)
    s = sim1(c, (0, 0, R + 1e-7), v=(V * math.sin(a), 0, -V * math.cos(a)), R=R, walls=FLOOR)
    fn, ft = [], []
    for _ in range(5000):
        s.step(1)
        F, _ = s.forces()
        fn.append(abs(F[0, 2]))
        ft.append(np.hypot(F[0, 0], F[0, 1]))
    return np.array(fn), np.array(ft)


def test_coulomb_limit_invariant_and_continuity():
    # Set-up of the paper's tangential-force comparison (Sec. 4.1.3): d = 2 mm,
    # rho = 7850, Y = 200 GPa, nu = 0.3, mu = 0.3, impacts at 5, 25 and 65 degrees from
    # the normal; the Coulomb limit binds over a growing part of the contact.
    frac = []
    for angle in (5.0, 25.0, 65.0):
        fn, ft = oblique_impact(angle)
        on = np.nonzero(fn > 0)[0]
        ratio = ft[on] / (0.3 * fn[on])
        assert ratio.max() <= 1.0 + 1e-12                   # |F_t| <= mu |F_n| always
        frac.append(np.mean(ratio > 1.0 - 1e-12))
        # F_t has no jump at the stick/slip switches (the first steps of the contact are
        # excluded: the damping force ~ delta_n^{1/4} rises steeply there by design)
        jumps = np.abs(np.diff(ft[on]))[3:-3]
        assert jumps.max() < 0.03 * ft.max()
    assert frac[0] < 0.05 < 0.1 < frac[1] < frac[2] and frac[2] > 0.5, frac


def test_momentum_conserved_by_pair_forces():
    wl = workloads.lattice(n=343, seed=7, walls=False, gravity=(0, 0, 0), speed=0.2)
    wl.cfg["domain_lo"] = (-0.01, -0.01, -0.01)
    wl.cfg["domain_hi"] = (0.04, 0.04, 0.04)
    s = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius)
    m = 2500.0 * 4.0 / 3.0 * math.pi * wl.radius.astype(float) ** 3
    p0 = (m[:, None] * wl.v).sum(0)
    scale = (m[:, None] * np.abs(wl.v)).sum()
    s.step(1)
    assert s.stats()["n_touch"] > 300
    s.step(299)
    _, v, _, _ = s.state()
    p1 = (m[:, None] * v).sum(0)
    assert np.abs(p1 - p0).max() / scale < 1e-13


def energy(wl_cfg, x, v, w, R, walls):
    m = wl_cfg["density"] * 4.0 / 3.0 * math.pi * R ** 3
    I = 0.4 * m * R ** 2
    g = np.array(wl_cfg["gravity"])
    E = 0.5 * (m[:, None] * v * v).sum() + 0.5 * (I[:, None] * w * w).sum() - (m * (x @ g)).sum()
    pm = wl_cfg["particle"]
    n = len(R)
    dx = x[None, :, :] - x[:, None, :]
    d = np.sqrt((dx ** 2).sum(-1))
    iu = np.triu_indices(n, 1)
    ov = (R[:, None] + R[None, :])[iu] - d[iu]
    Re = (R[:, None] * R[None, :] / (R[:, None] + R[None, :]))[iu]
    K = 4.0 / 3.0 * estar(pm, pm) * np.sqrt(Re)
    sel = ov > 0
    E += (0.4 * K[sel] * ov[sel] ** 2.5).sum()
    Kw = 4.0 / 3.0 * estar(pm, wl_cfg["wall"]) * np.sqrt(R)
    for wall in walls:
        nrm = np.array(wall["normal"]) / np.linalg.norm(wall["normal"])
        dist = (x - np.array(wall["point"])) @ nrm
        o = R - dist
        sel = o > 0
        E += (0.4 * Kw[sel] * o[sel] ** 2.5).sum()
    return E


def test_energy_conserved_without_dissipation():
    drifts = []
    for dt in (4e-6, 2e-6):
        wl = workloads.lattice(n=216, seed=11, spacing=1.05, speed=0.3, spin=0.0)
        for m in (wl.cfg["particle"], wl.cfg["wall"]):
            m.update(restitution=1.0, mu_slide=0.0, mu_roll=0.0)
        wl.cfg["dt"] = dt
        s = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
        R = wl.radius.astype(float)
        E0 = energy(wl.cfg, wl.x, wl.v, wl.w, R, wl.walls)
        m = 2500.0 * 4.0 / 3.0 * math.pi * R ** 3
        ke0 = 0.5 * (m[:, None] * wl.v ** 2).sum()
        worst = 0.0
        for _ in range(10):
            s.step(int(round(0.004 / dt / 10)))
            x, v, w, _ = s.state()
            worst = max(worst, abs(energy(wl.cfg, x, v, w, R, wl.walls) - E0) / ke0)
        assert s.stats()["n_touch"] > 0
        drifts.append(worst)
    assert drifts[0] < 1e-3
    assert drifts[1] < drifts[0] / 2.5        # second order in dt


def test_velocity_verlet_second_order_on_contact_oscillation():
    pm = mat(restitution=1.0)
    R = f32(1.5e-3)
    K = 4.0 / 3.0 * estar(pm, pm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    T = 2e-4

    def z_at(dt):
        c = cfg(particle=pm, wall=pm, dt=dt)
        s = sim1(c, (0, 0, R - 0.5 * d_eq), R=R, walls=FLOOR)
        s.step(int(round(T / dt)))
        x, _, _, _ = s.state()
        return x[0, 2]

    ref = z_at(2e-6 / 64)
    errs = [abs(z_at(dt) - ref) for dt in (2e-6, 1e-6, 5e-7)]
    orders = [math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])]
    assert all(abs(o - 2.0) < 0.15 for o in orders), orders


def numpy_pairs(x, rc, active=None):
    n = len(x)
    out = []
    for i in range(n):
        d = x[i + 1:] - x[i]
        s = d[:, 0] * d[:, 0]
        s = s + d[:, 1] * d[:, 1]
        s = s + d[:, 2] * d[:, 2]
        js = np.nonzero(s < rc * rc)[0] + i + 1
        for j in js:
            if active is None or (active[i] and active[j]):
                out.append((i, j))
    return np.array(out, dtype=np.int32).reshape(-1, 2)


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_cell_search_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 1500
    L = 0.03
    x = rng.uniform(0, L, (n, 3))
    R = rng.uniform(0.5e-3, 1e-3, n).astype(np.float32)
    rc = 1.3 * 2 * float(R.max())
    # adversarial pairs: exactly at the threshold distance, and one ulp either side
    for k, f in enumerate([1.0, 1.0 - 2 ** -52, 1.0 + 2 ** -52, 1.0 - 2 ** -50, 1.0 + 2 ** -50]):
        x[2 * k + 1] = x[2 * k] + np.array([rc * f, 0.0, 0.0])
    c = cfg(domain_lo=(0, 0, 0), domain_hi=(L, L, L), gravity=(0, 0, 0))
    s = oracle.OracleSim(c, x, np.zeros((n, 3)), np.zeros((n, 3)), R)
    got = s.pairs()
    ref = numpy_pairs(x, rc)
    assert got.shape == ref.shape and np.array_equal(got, ref)
    assert np.array_equal(oracle.brute_pairs(x, rc), ref)


def test_cell_search_outside_domain_is_clamped_correctly():
    rng = np.random.default_rng(9)
    n = 600
    x = rng.uniform(-0.01, 0.04, (n, 3))     # many outside the grid box [0, 0.03]^3
    R = np.full(n, 1e-3, np.float32)
    c = cfg(domain_lo=(0, 0, 0), domain_hi=(0.03, 0.03, 0.03), gravity=(0, 0, 0))
    s = oracle.OracleSim(c, x, np.zeros((n, 3)), np.zeros((n, 3)), R)
    assert np.array_equal(s.pairs(), numpy_pairs(x, 1.3 * 2e-3))


def test_dynamic_rebuild_keeps_all_contacts_in_list():
    # With skin, every touching pair must be in the fine-search list at every step.
    wl = workloads.lattice(n=216, seed=3, spacing=1.02, speed=0.5)
    wl.cfg["skin"] = 0.2 * 3e-3
    s = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
    R = wl.radius.astype(float)
    for _ in range(20):
        s.step(25)
        x, _, _, _ = s.state()
        touching = numpy_pairs(x, 2 * float(R.max()))
        lst = {tuple(p) for p in s.pairs()}
        assert all(tuple(p) in lst for p in touching)
    assert s.stats()["rebuilds"] > 2


def test_history_round_trip_resumes_identically():
    wl = workloads.lattice(n=125, seed=5, spacing=1.0, speed=0.3)
    a = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
    a.step(100)
    x, v, w, act = a.state()
    pairs, dtp, dtw = a.history()
    a.step(50)
    b = oracle.OracleSim(wl.cfg, x, v, w, wl.radius, wl.walls)
    b.set_history(pairs, dtp, dtw)
    b.step(50)
    xa, _, _, _ = a.state()
    xb, _, _, _ = b.state()
    # restarting from full-step velocities recomputes the forces at v^n instead of
    # v^{n-1/2}: the trajectories agree closely but not bitwise
    assert np.abs(xa - xb).max() < 1e-6


@pytest.mark.parametrize("poly", [0.0, 0.3])
def test_angular_momentum_changes_only_by_the_overlap_lever(poly):
    # Pair forces act along the centre line except F_t, whose torques R_i n x F_t and
    # R_j n x F_t act at the two surfaces; the rolling torques are +M_r and -M_r.  The total
    # L = sum m x x v + I w therefore changes only by delta_n n x F_t per contact (lever of
    # the overlap; velocity Verlet adds nothing for central forces), a fraction ~delta_n/R
    # of the spin changes.  A reversed or halved torque on either side changes L by a
    # fraction of order one of the tangential or rolling angular impulse; with unequal
    # radii, so does a lever taken from the wrong sphere.
    wl = workloads.lattice(n=343, seed=7, walls=False, gravity=(0, 0, 0), speed=0.2, poly=poly)
    wl.cfg["domain_lo"] = (-0.01, -0.01, -0.01)
    wl.cfg["domain_hi"] = (0.04, 0.04, 0.04)
    for m_ in (wl.cfg["particle"], wl.cfg["wall"]):
        m_["young"] = 1e8                  # small overlaps: a short lever
    wl.cfg["dt"] = 4e-6
    R = wl.radius.astype(float)
    m = 2500.0 * 4.0 / 3.0 * math.pi * R ** 3
    inertia = 0.4 * m * R ** 2

    def ang(x, v, w):
        return (m[:, None] * np.cross(x, v)).sum(0) + (inertia[:, None] * w).sum(0)

    s = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius)
    L0 = ang(wl.x, wl.v, wl.w)
    s.step(1)
    if poly == 0.0:
        assert s.stats()["n_touch"] > 100        # a touching lattice
    s.step(749)
    x, v, w, _ = s.state()
    spin_change = np.linalg.norm(inertia[:, None] * (w - wl.w), axis=1).sum()
    assert spin_change > 0.5 * np.linalg.norm(inertia[:, None] * wl.w, axis=1).sum()   # torques acted
    assert np.linalg.norm(ang(x, v, w) - L0) < 3e-3 * spin_change


def test_trajectory_is_independent_of_the_search_cadence():
    # A pair enters the force sum only while it touches, in list order (i < j, sorted), and
    # its tangential overlap survives a search; so a dynamic search with a thin or a thick
    # skin and a search at every step must give the same bits.  A lost overlap, or a
    # search that fires too late and misses a contact, breaks the equality.
    def run(**kw):
        wl = workloads.lattice(n=343, seed=21, spacing=1.0, speed=0.3)
        wl.cfg.update(kw)
        s = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
        s.step(3000)
        x, v, w, act = s.state()
        st = s.stats()
        s.close()
        return x.tobytes() + v.tobytes() + w.tobytes() + act.tobytes(), st

    thin, s_thin = run(skin=0.1 * 3e-3)
    thick, s_thick = run(skin=0.4 * 3e-3)
    every, s_every = run(skin=0.0, neighbor_factor=1.05, rebuild_every=1)
    assert s_every["rebuilds"] > s_thin["rebuilds"] > s_thick["rebuilds"] > 2
    assert s_thin["n_touch"] > 20
    assert thin == thick == every


def test_particles_leave_below_z_sink_and_stay_put():
    # Free fall is exact under velocity Verlet, z_n = z0 - g (n dt)^2 / 2, so the step at
    # which the centre first drops below z_sink is known; z_sink sits halfway between the
    # heights of that step and the one before, far from any rounding.
    dt, z0 = 1e-5, 0.05
    n_star = 1500
    z_before = z0 - 0.5 * G * ((n_star - 1) * dt) ** 2
    z_at = z0 - 0.5 * G * (n_star * dt) ** 2
    c = cfg(dt=dt, z_sink=0.5 * (z_before + z_at))
    s = sim1(c, (0.0, 0.0, z0))
    s.step(n_star - 1)
    assert s.state()[3][0] == 1
    s.step(1)
    x, _, _, act = s.state()
    assert act[0] == 0 and abs(x[0, 2] - z_at) < 1e-12
    s.step(200)
    x2, _, _, act2 = s.state()
    assert act2[0] == 0 and np.array_equal(x2, x)


def test_a_removed_particle_exerts_no_force():
    # A sits just above z_sink and leaves at the first drift; B starts 0.1 d above contact
    # with A, in A's fine-search list (skin 0.5 d), and falls through the place where A was
    # frozen before it has moved far enough to trigger a new search: B's fall stays the
    # exact free fall, whereas a pair term for the removed A would throw B back up.
    R = f32(1.5e-3)
    d = 2 * R
    dt = 1e-5
    zA = 0.0
    c = cfg(dt=dt, z_sink=zA - 1e-12, skin=0.5 * d)
    x = np.array([[0.0, 0.0, zA], [0.0, 0.0, zA + 1.1 * d]])
    s = oracle.OracleSim(c, x, np.zeros((2, 3)), np.zeros((2, 3)), np.array([R, R], np.float32))
    assert s.pairs().tolist() == [[0, 1]]
    steps = 1000                      # B falls 4.9e-4 m: past A's top, less than skin / 2
    s.step(steps)
    xs, _, _, act = s.state()
    t = steps * dt
    assert act.tolist() == [0, 1]
    assert xs[1, 2] < xs[0, 2] + 0.95 * d                      # B has reached A's place
    assert abs(xs[1, 2] - (zA + 1.1 * d - 0.5 * G * t * t)) < 1e-12
    assert s.stats()["rebuilds"] == 1


@pytest.mark.parametrize("every", [1, 7, 50])
def test_constant_search_runs_every_n_steps(every):
    # Sec. 3.1's constant mode: a search before the first step, then one every n steps
    wl = workloads.lattice(n=125, seed=2, spacing=1.0, speed=0.3)
    wl.cfg.update(skin=0.0, neighbor_factor=1.3, rebuild_every=every)
    s = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
    s.step(349)
    assert s.stats()["rebuilds"] == 1 + 349 // every


def spin_collision(w_i, w_j, mu, mu_r, v_rel=1.0, steps_per_tc=2000):
    """Head-on elastic collision of two equal steel spheres along x, spinning about z with
    w_i and w_j.  Returns R, m and the velocities and spins before and after."""
    R = f32(1e-3)
    m = mat(young=2e11, poisson=0.3, restitution=1.0, mu_slide=mu, mu_roll=mu_r)
    rho = 7850.0
    me = mass(R, rho) / 2.0
    K = 4.0 / 3.0 * estar(m, m) * math.sqrt(R / 2.0)
    dmax = (5.0 * me * v_rel ** 2 / (4.0 * K)) ** 0.4
    dt = 2.94328 * dmax / v_rel / steps_per_tc
    gap = 0.5 * v_rel * dt * 10
    x = np.array([[-R - gap, 0.0, 0.0], [R + gap, 0.0, 0.0]])
    v = np.array([[0.5 * v_rel, 0, 0], [-0.5 * v_rel, 0, 0]])
    w = np.array([[0, 0, w_i], [0, 0, w_j]], float)
    c = cfg(particle=m, wall=m, density=rho, gravity=(0, 0, 0), dt=dt, rolling_model=1,
            domain_lo=(-0.01, -0.01, -0.01), domain_hi=(0.01, 0.01, 0.01))
    s = oracle.OracleSim(c, x, v, w, np.array([R, R], np.float32))
    s.step(10 + steps_per_tc // 2)                 # half-way through the contact
    scales = s.force_scales()
    s.step(3 * steps_per_tc - 10 - steps_per_tc // 2)
    _, v1, w1, _ = s.state()
    spin_collision.mid_contact_scales = scales
    return R, mass(R, rho), v, w, v1, w1


def test_meshing_spins_do_not_slip_and_feel_only_rolling_resistance():
    # Opposite spins about z: the contact points move together, (R_i w_i + R_j w_j) x n = 0,
    # so there is no tangential force at all; the constant rolling torque -mu_r R_e |F_n|
    # w_ij/|w_ij| (w_ij = w_i - w_j) acts on i, its opposite on j.  Every force evaluation
    # pushes i along -x by |F_n| and turns it by mu_r R_e |F_n|, so over the collision
    # I dw_i = mu_r R_e m dv_x,i exactly.
    mu_r = 0.1
    R, m, v0, w0, v1, w1 = spin_collision(1000.0, -1000.0, 0.3, mu_r)
    inertia = 0.4 * m * R * R
    dvx = v1[0, 0] - v0[0, 0]
    assert abs(dvx + 1.0) < 1e-6                           # elastic: the spheres swap velocities
    assert np.all(v1[:, 1:] == 0.0)                        # no tangential force
    dw_i = w1[0, 2] - w0[0, 2]
    assert abs(dw_i - mu_r * (R / 2) * m * dvx / inertia) < 1e-12 * abs(dw_i)
    assert abs((w1[1, 2] - w0[1, 2]) + dw_i) < 1e-12 * abs(dw_i)
    # the error scales mid-contact: |M| = mu_r R_e |F| on both spheres (no tangential force)
    Fa, Ma = spin_collision.mid_contact_scales
    assert Fa[0] > 0.0 and Fa[1] == Fa[0]
    assert np.allclose(Ma, mu_r * (R / 2) * Fa, rtol=1e-12, atol=0)


def test_sliding_collision_tangential_impulse_is_mu_times_normal():
    # Equal spins about z: the contact points slide past each other at 2 R w, fast enough
    # to keep sliding through the whole collision, so |F_t| = mu |F_n| at every evaluation
    # and F_t on i opposes the slip (-y).  Hence dv_y,i = mu dv_x,i, dv_y,j = -dv_y,i, and
    # both spins slow by R mu m |dv_x| / I = 2.5 mu |dv_x| / R (up to the small turn of the
    # centre line during the collision).
    mu = 0.3
    R, m, v0, w0, v1, w1 = spin_collision(2000.0, 2000.0, mu, 0.0)
    dvx = v1[0, 0] - v0[0, 0]
    dvy = v1[0, 1] - v0[0, 1]
    assert dvx < -0.99
    assert abs(dvy - mu * dvx) < 5e-3 * mu * abs(dvx)
    assert v1[1, 1] == -v1[0, 1]
    for k in range(2):
        assert abs((w1[k, 2] - w0[k, 2]) - 2.5 * mu * dvx / R) < 5e-3 * 2.5 * mu * abs(dvx) / R
    assert 2 * R * w1[0, 2] + (v1[0, 1] - v1[1, 1]) > 0.0      # still sliding at the end


def test_error_scales_of_a_sliding_sphere():
    # The per-particle error scales (sum of |contact force| and of |contact torque|, used to
    # normalise the GPU force errors) of a sphere sliding on a floor under the Coulomb
    # limit with constant rolling resistance: |F| = N sqrt(1 + mu^2) and
    # |M| = R mu N + mu_r R N with N = m g (R_e = R against a wall), every evaluation anew.
    mu, mu_r = 0.3, 0.1
    wm = mat(restitution=0.5, mu_slide=mu, mu_roll=mu_r)
    R = f32(1.5e-3)
    c = cfg(wall=wm, particle=mat(restitution=0.5), dt=2e-6, rolling_model=1)
    K = 4.0 / 3.0 * estar(c["particle"], wm) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    s = sim1(c, (0, 0, R - d_eq), v=(0.2, 0, 0), w=(0, 5.0, 0), R=R, walls=FLOOR)
    for _ in range(3):
        s.step(500)                              # well inside the sliding phase
        Fa, Ma = s.force_scales()
        N = mass(R) * G
        assert abs(Fa[0] - N * math.sqrt(1 + mu * mu)) < 1e-3 * N
        assert abs(Ma[0] - (R * mu * N + mu_r * R * N)) < 1e-3 * R * N


def test_wall_contacts_are_invariant_under_translation():
    # Moving a wall (its point and rotation origin) and the sphere by the same vector must
    # not change the contact force or torque: a plane, a spinning drum wall touched away
    # from the axis origin, and an annulus touched on its face and on its rim.
    pm = mat(restitution=0.5, mu_roll=0.1)
    wm = mat(restitution=0.5, young=3e7, mu_roll=0.1)
    R = f32(2.5e-3)
    c = cfg(particle=pm, wall=wm, gravity=(0, 0, 0), domain_lo=(-0.2, -0.2, -0.2), domain_hi=(0.2, 0.2, 0.2))
    Rc = 0.05
    cases = [
        (lambda o: [workloads.plane(o, (0, 0, 1))], (0.01, -0.02, 2.3e-3)),
        (lambda o: [workloads.cylinder(o, (0, 1, 0), Rc, omega=3.0, rot_origin=o, rot_axis=(0, 1, 0))],
         (0.03, 0.017, -math.sqrt((Rc - R + 2e-4) ** 2 - 0.03 ** 2))),
        (lambda o: [workloads.annulus(o, (0, 0, 1), 0.5, 0.004)], (0.02, 0.0, 2.4e-3)),
        (lambda o: [workloads.annulus(o, (0, 0, 1), 0.5, 0.004)], (0.0025, 0.001, 1.5e-3)),
    ]
    offset = np.array([0.013, -0.021, 0.034])
    for make, p in cases:
        out = []
        for o in (np.zeros(3), offset):
            s = sim1(c, tuple(np.array(p) + o), v=(0.1, -0.2, 0.05), w=(3.0, -1.0, 2.0), R=R,
                     walls=make(tuple(o)))
            F, M = s.forces()
            out.append((F[0], M[0]))
        (F0, M0), (F1, M1) = out
        assert np.linalg.norm(F0) > 0.0
        assert np.allclose(F1, F0, rtol=1e-8, atol=1e-8 * np.linalg.norm(F0))
        assert np.allclose(M1, M0, rtol=1e-8, atol=1e-8 * np.linalg.norm(M0) + 1e-30)
    # and at rest, away from the axis origin, a still drum wall pushes towards its axis
    # with the Hertz force of the 0.2 mm overlap (R_e = R: a wall of infinite radius)
    p = np.array(cases[1][1]) + offset
    s = sim1(c, tuple(p), R=R, walls=[workloads.cylinder(tuple(offset), (0, 1, 0), Rc)])
    F, _ = s.forces()
    radial = np.array([p[0] - offset[0], 0.0, p[2] - offset[2]])
    K = 4.0 / 3.0 * estar(pm, wm) * math.sqrt(R)
    expect = -K * 2e-4 ** 1.5 * radial / np.linalg.norm(radial)
    assert np.allclose(F[0], expect, rtol=1e-6, atol=1e-9 * np.linalg.norm(expect))


def test_cell_search_with_an_offset_domain_equals_brute_force():
    rng = np.random.default_rng(4)
    n = 1200
    lo = np.array([-0.013, 0.007, -0.021])
    L = 0.03
    x = lo + rng.uniform(0, L, (n, 3))
    R = rng.uniform(0.5e-3, 1e-3, n).astype(np.float32)
    rc = 1.3 * 2 * float(R.max())
    c = cfg(domain_lo=tuple(lo), domain_hi=tuple(lo + L), gravity=(0, 0, 0))
    s = oracle.OracleSim(c, x, np.zeros((n, 3)), np.zeros((n, 3)), R)
    assert np.array_equal(s.pairs(), numpy_pairs(x, rc))


def test_spheres_that_never_meet_move_as_if_alone():
    # Superposition: three spheres far apart, each sliding and spinning on the same floor,
    # follow exactly the trajectories they have alone -- per-particle state, wall contacts
    # and their tangential overlaps do not leak between particles.
    R = f32(1.5e-3)
    c = cfg(wall=mat(restitution=0.5, mu_slide=0.3, mu_roll=0.1), dt=2e-6)
    # a tilted floor, so that the tangential overlaps have all three components
    nrm = np.array([0.3, -0.2, 1.0]) / np.linalg.norm([0.3, -0.2, 1.0])
    floor = [workloads.plane((0, 0, 0), tuple(nrm))]
    base = np.array([[-0.05, 0.0, 0.0], [0.0, 0.04, 0.0], [0.05, -0.03, 0.0]])
    K = 4.0 / 3.0 * estar(c["particle"], c["wall"]) * math.sqrt(R)
    d_eq = (mass(R) * G * nrm[2] / K) ** (2.0 / 3.0)       # resting overlap on the slope
    x = base - (base @ nrm)[:, None] * nrm + (R - d_eq) * nrm
    v = np.array([[0.2, 0.0, 0.0], [0.0, -0.15, 0.0], [0.1, 0.1, 0.0]])
    v = v - (v @ nrm)[:, None] * nrm
    w = np.array([[0.0, 30.0, 0.0], [40.0, 0.0, 5.0], [-20.0, 10.0, 0.0]])
    together = oracle.OracleSim(c, x, v, w, np.full(3, R, np.float32), floor)
    together.step(3000)
    xt, vt, wt, _ = together.state()
    assert together.stats()["n_wall_touch"] == 3
    for k in range(3):
        alone = sim1(c, tuple(x[k]), v=tuple(v[k]), w=tuple(w[k]), R=R, walls=floor)
        alone.step(3000)
        xa, va, wa, _ = alone.state()
        assert np.array_equal(xa[0], xt[k]) and np.array_equal(va[0], vt[k]) and np.array_equal(wa[0], wt[k])


def test_translating_turntable_carries_a_co_moving_sphere():
    # A plate that slides along x at V while spinning about the vertical axis through a
    # point that moves with it: a sphere resting on the axis with the plate's velocity and
    # spin has no slip and no relative spin, so it rides along at V without drifting.
    R = f32(1.5e-3)
    V, Om = 0.05, 4.0
    c = cfg(wall=mat(restitution=0.5, mu_slide=0.3, mu_roll=0.1), dt=2e-6)
    K = 4.0 / 3.0 * estar(c["particle"], c["wall"]) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    plate = [workloads.plane((0, 0, 0), (0, 0, 1), omega=Om, rot_origin=(0.01, 0, 0), rot_axis=(0, 0, 1),
                             velocity=(V, 0, 0), translates=1)]
    s = sim1(c, (0.01, 0.0, R - d_eq), v=(V, 0, 0), w=(0, 0, Om), R=R, walls=plate)
    steps = 5000
    s.step(steps)
    x, v, w, _ = s.state()
    t = steps * 2e-6
    # rounding of x against the moving axis leaves a slip of ~1e-9 m/s: drift of ~1e-8 m
    # (an axis left behind at -V t would drag the sphere sideways by ~Om V t^2 = 2e-5 m)
    assert abs(x[0, 0] - (0.01 + V * t)) < 1e-8 and abs(x[0, 1]) < 1e-7
    assert abs(v[0, 0] - V) < 1e-5 and abs(v[0, 1]) < 1e-5
    assert abs(w[0, 2] - Om) < 1e-6


def test_floating_wall_window_is_half_open():
    # A floating wall acts for t_on <= t < t_off (reading of Sec. 3.6).  dt = 2^-16 s makes
    # both times exact: a falling sphere meets a wall that appears at t_on under it, and a
    # sphere resting on a wall that vanishes at t_off is supported one step before and not
    # at t_off.
    R = f32(1.5e-3)
    dt = 2.0 ** -16
    c = cfg(particle=mat(restitution=0.3), wall=mat(restitution=0.3), dt=dt)
    appears = [workloads.plane((0, 0, 0), (0, 0, 1), t_on=50 * dt)]
    s = sim1(c, (0, 0, R - 1e-6), R=R, walls=appears)
    assert s.forces()[0][0, 2] == 0.0       # t = 0 < t_on
    s.step(49)
    assert s.forces()[0][0, 2] == 0.0       # t = 49 dt
    s.step(1)
    assert s.forces()[0][0, 2] > 0.0        # t = t_on: present
    K = 4.0 / 3.0 * estar(c["particle"], c["wall"]) * math.sqrt(R)
    d_eq = (mass(R) * G / K) ** (2.0 / 3.0)
    vanishes = [workloads.plane((0, 0, 0), (0, 0, 1), t_off=100 * dt)]
    s = sim1(c, (0, 0, R - d_eq), R=R, walls=vanishes)
    s.step(99)
    assert s.forces()[0][0, 2] > 0.5 * mass(R) * G      # t = 99 dt: holding the sphere
    s.step(1)
    assert s.forces()[0][0, 2] == 0.0       # t = t_off: gone


def rotation(axis, angle):
    """Rotation matrix about `axis` (Rodrigues)."""
    k = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


Q = rotation((0.3, -0.5, 0.8), 1.1)


def test_an_oblique_spinning_collision_is_rotation_invariant():
    # Rotating the whole system rotates the result: three spheres (a far spectator first,
    # so the colliding pair is (1, 2)), an oblique collision with spins and sliding
    # friction, and constant rolling resistance, run as given and rotated by Q.
    R = f32(1e-3)
    m = mat(young=2e11, poisson=0.3, restitution=0.7, mu_slide=0.3, mu_roll=0.1)
    c = cfg(particle=m, wall=m, density=7850.0, gravity=(0, 0, 0), dt=2e-8,
            domain_lo=(-0.02, -0.02, -0.02), domain_hi=(0.02, 0.02, 0.02))
    x = np.array([[0.012, -0.011, 0.01], [-1.05e-3, 0.0, 0.0], [1.05e-3, 4e-4, -2e-4]])
    v = np.array([[0.0, 0.0, 0.0], [0.5, 0.1, -0.05], [-0.5, 0.05, 0.1]])
    w = np.array([[0.0, 0.0, 0.0], [300.0, -200.0, 500.0], [-100.0, 400.0, 250.0]])
    out = []
    for T in (np.eye(3), Q):
        s = oracle.OracleSim(c, x @ T.T, v @ T.T, w @ T.T, np.full(3, R, np.float32))
        s.step(1)
        assert s.stats()["n_touch"] == 0
        s.step(9999)
        xs, vs, ws, _ = s.state()
        out.append((xs, vs, ws))
    (x0, v0, w0), (x1, v1, w1) = out
    assert np.abs(v0[1:] - v[1:]).max() > 0.05 and np.abs(w0[1:] - w[1:]).max() > 10.0   # they collided
    assert np.allclose(x1, x0 @ Q.T, rtol=0, atol=1e-12)
    assert np.allclose(v1, v0 @ Q.T, rtol=0, atol=1e-9)
    assert np.allclose(w1, w0 @ Q.T, rtol=0, atol=1e-6)


def test_wall_contacts_are_rotation_invariant():
    # A plane, a drum wall spinning about its axis, and an annulus (face and rim), each
    # with the sphere and all wall vectors rotated by Q and moved off the origin: the
    # force and torque rotate with them.
    pm = mat(restitution=0.5, mu_roll=0.1)
    wm = mat(restitution=0.5, young=3e7, mu_roll=0.1)
    R = f32(2.5e-3)
    c = cfg(particle=pm, wall=wm, gravity=(0, 0, 0), domain_lo=(-0.2, -0.2, -0.2), domain_hi=(0.2, 0.2, 0.2))
    Rc = 0.05
    off = np.array([0.013, -0.021, 0.034])

    def walls(T, o):
        y, z = T @ np.array([0.0, 1.0, 0.0]), T @ np.array([0.0, 0.0, 1.0])
        o = tuple(o)
        return [
            [workloads.plane(o, tuple(z))],
            [workloads.cylinder(o, tuple(y), Rc, omega=3.0, rot_origin=o, rot_axis=tuple(y))],
            [workloads.annulus(o, tuple(z), 0.5, 0.004, omega=-2.0, rot_origin=o, rot_axis=tuple(z))],
            [workloads.annulus(o, tuple(z), 0.5, 0.004)],
        ]

    spots = [(0.01, -0.02, 2.3e-3), (0.03, 0.017, -math.sqrt((Rc - R + 2e-4) ** 2 - 0.03 ** 2)),
             (0.02, 0.0, 2.4e-3), (0.0025, 0.001, 1.5e-3)]
    v, w = np.array([0.1, -0.2, 0.05]), np.array([3.0, -1.0, 2.0])
    for k, p in enumerate(spots):
        res = []
        for T, o in ((np.eye(3), np.zeros(3)), (Q, off)):
            s = sim1(c, tuple(T @ np.array(p) + o), v=tuple(T @ v), w=tuple(T @ w), R=R, walls=walls(T, o)[k])
            F, M = s.forces()
            res.append((F[0], M[0]))
        (F0, M0), (F1, M1) = res
        assert np.linalg.norm(F0) > 0.0
        assert np.allclose(F1, Q @ F0, rtol=0, atol=1e-8 * np.linalg.norm(F0)), k
        assert np.allclose(M1, Q @ M0, rtol=0, atol=1e-8 * np.linalg.norm(M0) + 1e-30), k


def test_sphere_on_the_axis_of_the_orifice_touches_the_whole_rim():
    # Centred over the hole, every rim point is nearest: whichever the contact takes, its
    # overlap is R - sqrt(r_in^2 + h^2) and the force has that Hertz magnitude.
    pm = mat(restitution=1.0)
    wm = mat(restitution=1.0, young=3e7)
    R = f32(2.5e-3)
    r_in, h = 0.002, 1.2e-3
    # (exactly on the axis: a plate in the xy plane through the origin, so that the in-plane
    # offset is exactly zero; off the origin or tilted, rounding leaves a spurious offset
    # whose direction is not in the plate)
    c = cfg(particle=pm, wall=wm, gravity=(0, 0, 0))
    s = sim1(c, (0.0, 0.0, h), R=R, walls=[workloads.annulus((0, 0, 0), (0, 0, 1), 0.5, r_in)])
    F, _ = s.forces()
    K = 4.0 / 3.0 * estar(pm, wm) * math.sqrt(R)
    delta = R - math.hypot(r_in, h)
    assert abs(np.linalg.norm(F[0]) - K * delta ** 1.5) < 1e-9 * K * delta ** 1.5
    assert abs(F[0, 2] - K * delta ** 1.5 * h / math.hypot(r_in, h)) < 1e-9 * K * delta ** 1.5


def test_a_paddle_turning_about_its_contact_point_does_not_drag():
    # A vertical plate (normal +x) turning about the vertical axis through the point the
    # sphere touches: the surface does not move there, so a still sphere feels only the
    # normal force, although the plate spins.
    R = f32(1.5e-3)
    c = cfg(gravity=(0, 0, 0))
    paddle = [workloads.plane((0, 0, 0), (1, 0, 0), omega=5.0, rot_origin=(0, 0, 0), rot_axis=(0, 0, 1))]
    s = sim1(c, (R - 1e-5, 0.0, 0.0), R=R, walls=paddle)
    F, M = s.forces()
    assert F[0, 0] > 0.0 and F[0, 1] == 0.0 and F[0, 2] == 0.0
    assert np.all(M[0] == 0.0)


def test_restart_from_saved_state_and_overlaps_reproduces_the_forces():
    # With e = 1 and no rolling resistance the contact law depends only on positions and
    # tangential overlaps.  A new simulation given a saved state and the saved
    # particle-particle and particle-wall overlaps reads them back unchanged and, at its
    # first evaluation (new-1: no overlap increment), finds the forces the original
    # evaluated last (to rounding: the Coulomb limit is re-applied to the saved overlap).
    wl = workloads.lattice(n=216, seed=8, spacing=0.995, speed=0.05, spin=5.0)
    settle = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
    settle.step(3000)                           # a bed resting on the floor and the walls
    x0, v0, w0, _ = settle.state()
    p0, h0, hw0 = settle.history()
    c = dict(wl.cfg, particle=dict(wl.cfg["particle"], restitution=1.0, mu_roll=0.0),
             wall=dict(wl.cfg["wall"], restitution=1.0, mu_roll=0.0))
    a = oracle.OracleSim(c, x0, v0, w0, wl.radius, wl.walls)
    a.set_history(p0, h0, hw0)
    a.step(50)
    x, v, w, act = a.state()
    Fa, Ma = a.forces()
    scale_f, scale_m = a.force_scales()
    pairs, dtp, dtw = a.history()
    assert len(pairs) > 10 and np.count_nonzero(dtw) > 0
    b = oracle.OracleSim(c, x, v, w, wl.radius, wl.walls)
    b.set_history(pairs, dtp, dtw)
    pb, hb, hwb = b.history()                   # (reading them runs the first evaluation)
    assert np.array_equal(pb, pairs)
    assert np.allclose(hb, dtp, rtol=1e-12, atol=0) and np.allclose(hwb, dtw, rtol=1e-12, atol=0)
    Fb, Mb = b.forces()
    assert np.all(np.linalg.norm(Fb - Fa, axis=1) <= 1e-12 * (scale_f + 1e-30))
    assert np.all(np.linalg.norm(Mb - Ma, axis=1) <= 1e-12 * (scale_m + 1e-30))


def test_forces_of_many_particles_obey_newtons_third_law():
    # Pair forces only (no walls, no gravity): the forces read back for every particle sum
    # to zero up to rounding, and so do their moments about the origin up to the lever of
    # the overlaps.
    wl = workloads.lattice(n=343, seed=9, walls=False, gravity=(0, 0, 0), speed=0.3, spin=30.0)
    wl.cfg["domain_lo"] = (-0.01, -0.01, -0.01)
    wl.cfg["domain_hi"] = (0.04, 0.04, 0.04)
    s = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius)
    s.step(5)
    F, M = s.forces()
    Fa, _ = s.force_scales()
    assert s.stats()["n_touch"] > 300
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * Fa.sum()
    assert np.count_nonzero(np.linalg.norm(F, axis=1)) > 300


def test_set_state_round_trip_and_clock():
    wl = workloads.lattice(n=64, seed=3)
    s = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
    rng = np.random.default_rng(1)
    x2, v2, w2 = wl.x + 1e-5 * rng.normal(size=wl.x.shape), rng.normal(size=(64, 3)), rng.normal(size=(64, 3))
    s.set_state(x2, v2, w2)
    x, v, w, act = s.state()
    assert np.array_equal(x, x2) and np.array_equal(v, v2) and np.array_equal(w, w2) and act.all()
    s.step(37)
    st = s.stats()
    assert st["steps"] == 37 and st["time"] == 37 * wl.cfg["dt"] and st["n_active"] == 64
