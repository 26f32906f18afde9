"""Helpers shared by the GPU parity tests: run the same seeded input through the CUDA
library and through the CPU oracle, and measure their differences."""
import math

import numpy as np

import oracle
import workloads


def make_gpu(wl, precision, **kw):
    from paper_2106_09576_gb300 import DEM
    return DEM(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls, precision=precision, **kw)


def make_oracle(wl):
    return oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)


def masses(wl):
    R = wl.radius.astype(np.float64)
    return wl.cfg["density"] * 4.0 / 3.0 * math.pi * R ** 3


def force_error(F_gpu, F_ref, scale, m, g):
    """Per particle |F_gpu - F_ref| / (sum of |contact force| + m |g|), max over particles
    (the normalisation keeps particles whose contact forces cancel from dominating)."""
    den = scale + m * np.linalg.norm(g)
    return float(np.max(np.linalg.norm(F_gpu - F_ref, axis=1) / den))


def torque_error(M_gpu, M_ref, scale, m, R, g):
    den = scale + m * np.linalg.norm(g) * R
    return float(np.max(np.linalg.norm(M_gpu - M_ref, axis=1) / den))


def random_history(wl, pairs, seed, frac=0.7, scale=2e-6):
    """Non-zero tangential overlaps on a random subset of the given (touching) pairs."""
    rng = np.random.default_rng(seed)
    sel = rng.random(len(pairs)) < frac
    p = pairs[sel]
    vals = rng.normal(0.0, scale, (len(p), 3))
    return p, vals


def touching_pairs(x, R):
    n = len(x)
    out = []
    for i in range(n):
        d = np.linalg.norm(x[i + 1:] - x[i], axis=1)
        js = np.nonzero(d < R[i] + R[i + 1:])[0] + i + 1
        out.extend((i, j) for j in js)
    return np.array(out, dtype=np.int32).reshape(-1, 2)


def subsystem(x, R, sample, rc):
    """Indices of all particles within rc (plus margin) of the sampled particles."""
    keep = set(int(s) for s in sample)
    from scipy.spatial import cKDTree
    tree = cKDTree(x)
    for s in sample:
        keep.update(tree.query_ball_point(x[s], rc * 1.0001))
    idx = np.array(sorted(keep), dtype=np.int64)
    return idx
