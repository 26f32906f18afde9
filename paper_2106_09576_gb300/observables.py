"""Macroscopic observables of long rollouts, computed on the host from states.

Long DEM runs diverge chaotically, so two precisions (or the surrogate and plain DEM) are
compared through these quantities rather than trajectories: the silo discharge rate, the
packing fraction of a settled bed, the dynamic angle of repose of a rotating drum and the
kinetic energy."""
import math

import numpy as np


def discharge_rate(t, discharged, n0, lo=0.2, hi=0.8):
    """Particles per second: least-squares slope of the discharged count against time
    over the samples where between lo and hi of the initial n0 particles have left."""
    t = np.asarray(t, dtype=np.float64)
    d = np.asarray(discharged, dtype=np.float64)
    sel = (d >= lo * n0) & (d <= hi * n0)
    if sel.sum() < 3:
        raise ValueError("fewer than three samples inside the fitting window")
    A = np.vstack([t[sel], np.ones(sel.sum())]).T
    slope, _ = np.linalg.lstsq(A, d[sel], rcond=None)[0]
    return float(slope)


def packing_fraction(x, radius, active, R_wall, z_floor, d):
    """Solid fraction of a settled bed in a vertical cylinder of radius R_wall (axis on z
    through the origin) with its floor at z_floor: sphere volumes whose centres lie in a
    coaxial probe cylinder kept 3 d away from the wall, the floor and the free surface
    (the highest centre), divided by the probe volume."""
    x = np.asarray(x)[np.asarray(active, dtype=bool)]
    r = np.asarray(radius, dtype=np.float64)[np.asarray(active, dtype=bool)]
    top = float(x[:, 2].max())
    rp, z0, z1 = R_wall - 3 * d, z_floor + 3 * d, top - 3 * d
    if rp <= 0 or z1 <= z0:
        raise ValueError("bed too small for a probe 3 d from walls and surface")
    inside = (np.hypot(x[:, 0], x[:, 1]) < rp) & (x[:, 2] > z0) & (x[:, 2] < z1)
    vol = float(np.sum(4.0 / 3.0 * math.pi * r[inside] ** 3))
    return vol / (math.pi * rp * rp * (z1 - z0))


def angle_of_repose(x, radius, active, L, d_max, axis_origin_y=0.0):
    """Free-surface angle in degrees of a drum whose axis is the y axis (gravity along -z):
    in the central axial half (L/4 < y - y0 < 3L/4), the highest sphere top per bin of
    width 2 d_max along x; least-squares line through the middle 60 % of the occupied
    bins; the angle of its slope."""
    a = np.asarray(active, dtype=bool)
    x = np.asarray(x)[a]
    r = np.asarray(radius, dtype=np.float64)[a]
    y = x[:, 1] - axis_origin_y
    sel = (y > 0.25 * L) & (y < 0.75 * L)
    xs, top = x[sel, 0], x[sel, 2] + r[sel]
    w = 2.0 * d_max
    b = np.floor(xs / w).astype(np.int64)
    bins = np.unique(b)
    hx = np.array([(k + 0.5) * w for k in bins])
    hz = np.array([top[b == k].max() for k in bins])
    m = len(bins)
    k0, k1 = int(round(0.2 * m)), int(round(0.8 * m))
    if k1 - k0 < 3:
        raise ValueError("too few occupied bins")
    slope, _ = np.polyfit(hx[k0:k1], hz[k0:k1], 1)
    return float(math.degrees(math.atan(abs(slope))))


def kinetic_energy(v, w, radius, density, active=None):
    """Translational plus rotational kinetic energy of solid spheres (J)."""
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    r = np.asarray(radius, dtype=np.float64)
    m = density * 4.0 / 3.0 * math.pi * r ** 3
    e = 0.5 * m * (v * v).sum(1) + 0.5 * (0.4 * m * r * r) * (w * w).sum(1)
    if active is not None:
        e = e[np.asarray(active, dtype=bool)]
    return float(e.sum())
