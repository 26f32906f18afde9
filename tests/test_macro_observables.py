"""The macroscopic observables used to compare long rollouts, pinned on inputs whose
answer is known in closed form."""
import math

import numpy as np
import pytest

from macro import angle_of_repose, discharge_rate, packing_fraction


def test_discharge_rate_recovers_a_constant_flow():
    t = np.linspace(0.0, 2.0, 401)
    n0, rate, t0 = 10000, 7300.0, 0.3
    d = np.clip(np.floor(rate * (t - t0)), 0, n0)
    assert discharge_rate(t, d, n0) == pytest.approx(rate, rel=2e-3)
    # samples outside 20-80 % (start-up and the tail) do not bias the fit
    d2 = d.copy()
    d2[d2 < 0.2 * n0] *= 0.5
    d2[d2 > 0.8 * n0] = 0.8 * n0 + 1.0
    assert discharge_rate(t, d2, n0) == pytest.approx(rate, rel=2e-3)


def test_packing_fraction_of_a_simple_cubic_lattice():
    # spheres of diameter d on a cubic lattice of spacing a fill pi/6 (d/a)^3
    d, a = 2e-3, 2.2e-3
    m = 60
    g = (np.arange(m) - (m - 1) / 2.0) * a
    X, Y, Z = np.meshgrid(g, g, np.arange(m) * a + a / 2, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    R = 0.5 * m * a
    keep = np.hypot(x[:, 0], x[:, 1]) < R - 0.5 * d
    x = x[keep]
    r = np.full(len(x), 0.5 * d)
    phi = packing_fraction(x, r, np.ones(len(x), bool), R, 0.0, d)
    assert phi == pytest.approx(math.pi / 6 * (d / a) ** 3, rel=0.02)


@pytest.mark.parametrize("deg", [18.0, 27.0, 35.0])
def test_angle_of_repose_of_an_inclined_pile(deg):
    rng = np.random.default_rng(3)
    d, L = 4e-3, 0.05
    n = 20000
    x = np.empty((n, 3))
    x[:, 0] = rng.uniform(-0.1, 0.1, n)
    x[:, 1] = rng.uniform(0, L, n)
    surf = math.tan(math.radians(deg)) * x[:, 0]
    x[:, 2] = surf - rng.uniform(0, 0.05, n)
    # a dense skin of spheres on the surface plane
    k = 4000
    s = np.empty((k, 3))
    s[:, 0] = rng.uniform(-0.1, 0.1, k)
    s[:, 1] = rng.uniform(0, L, k)
    s[:, 2] = math.tan(math.radians(deg)) * s[:, 0]
    x = np.vstack([x, s])
    r = np.full(len(x), 0.5 * d)
    got = angle_of_repose(x, r, np.ones(len(x), bool), L, d)
    assert got == pytest.approx(deg, abs=0.5)
