"""Seeded synthetic DEM inputs shaped like the workloads of Lethe-DEM (arXiv 2106.09576).

This module only places spheres and writes configuration dicts; it holds none of the
method's arithmetic (no forces, no search, no integration).  Both the CUDA path and the
CPU oracle read its output, so neither depends on the other.

Every generator is seeded with NumPy ``Generator(PCG64)``; the default seed of a
workload is ``2106 + 1000 * config_index + instance``.

Shapes (the paper's experiments, whose data are not available, stand behind them):
  * ``cube``    -- 1,000 monodisperse spheres (d = 3 mm) placed at random without
                   overlap in a 0.1 m box with six plane walls (a settling test).
  * ``lattice`` -- the same box filled densely on a jittered lattice, slightly
                   compressed, with random velocities and spins, for one-step parity.
  * ``drum``    -- a rotating drum of polydisperse spheres (r in U[1.5, 2.5] mm),
                   horizontal axis, filled on an FCC lattice; the drum of the
                   rotating-drum validation case, scaled so 200k spheres fill half of it.
  * ``silo``    -- a flat-bottomed cylindrical silo (R = 0.5 m, orifice 0.05 m) of
                   monodisperse d = 5 mm spheres filled on a jittered cubic lattice,
                   plugged by a floating wall, like the 4.3M-particle packing case.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 2106


def seed_for(config_index: int, instance: int = 0) -> int:
    return BASE_SEED + 1000 * config_index + instance


def material(young=1e7, poisson=0.3, restitution=0.9, mu_slide=0.3, mu_roll=0.1) -> dict:
    return dict(young=young, poisson=poisson, restitution=restitution, mu_slide=mu_slide,
                mu_roll=mu_roll)


@dataclasses.dataclass
class Workload:
    name: str
    cfg: dict
    walls: list
    x: np.ndarray        # [n, 3] float64
    v: np.ndarray        # [n, 3] float64
    w: np.ndarray        # [n, 3] float64
    radius: np.ndarray   # [n] float32

    @property
    def n(self) -> int:
        return int(len(self.radius))


def plane(point, normal, **kw) -> dict:
    d = dict(kind=0, point=tuple(map(float, point)), normal=tuple(map(float, normal)))
    d.update(kw)
    return d


def cylinder(point, axis, radius, **kw) -> dict:
    d = dict(kind=1, point=tuple(map(float, point)), normal=tuple(map(float, axis)),
             radius=float(radius))
    d.update(kw)
    return d


def annulus(center, normal, outer, inner, **kw) -> dict:
    d = dict(kind=2, point=tuple(map(float, center)), normal=tuple(map(float, normal)),
             radius=float(outer), inner_radius=float(inner))
    d.update(kw)
    return d


def box_walls(lo, hi) -> list:
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    walls = []
    for a in range(3):
        n = np.zeros(3); n[a] = 1.0
        walls.append(plane(lo, n))
        walls.append(plane(hi, -n))
    return walls


def _base_cfg(**kw) -> dict:
    cfg = dict(density=2500.0, particle=material(), wall=material(), gravity=(0.0, 0.0, -9.81),
               dt=1e-5, neighbor_factor=1.3, skin=0.0, rebuild_every=0, rolling_model=1,
               z_sink=-1e300, precision="fp64")
    cfg.update(kw)
    return cfg


def _rsa(rng, n, r, lo, hi, max_tries=200):
    """Random sequential addition of n spheres of radius r in the box [lo+r, hi-r]."""
    lo = np.asarray(lo, float) + r
    hi = np.asarray(hi, float) - r
    h = 2.0 * r
    dims = np.maximum(1, np.floor((hi - lo) / h).astype(int))
    grid = {}
    out = np.empty((n, 3))
    k = 0
    tries = 0
    while k < n:
        p = lo + rng.random(3) * (hi - lo)
        c = tuple(np.minimum(dims - 1, ((p - lo) / h).astype(int)))
        ok = True
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    for q in grid.get((c[0] + dx, c[1] + dy, c[2] + dz), ()):
                        if np.sum((out[q] - p) ** 2) < (2.0 * r) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        tries += 1
        if tries > max_tries * n:
            raise RuntimeError("random sequential addition did not converge")
        if not ok:
            continue
        out[k] = p
        grid.setdefault(c, []).append(k)
        k += 1
    return out


def cube(n: int = 1000, seed: int | None = None, d: float = 3e-3, L: float = 0.1,
         precision: str = "fp64") -> Workload:
    """Random non-overlapping monodisperse spheres at rest in a closed box, gravity -z."""
    rng = np.random.Generator(np.random.PCG64(seed_for(0) if seed is None else seed))
    r = 0.5 * d
    x = _rsa(rng, n, r, (0, 0, 0), (L, L, L))
    cfg = _base_cfg(domain_lo=(0.0, 0.0, 0.0), domain_hi=(L, L, L), dt=1e-5, precision=precision)
    return Workload("cube", cfg, box_walls((0, 0, 0), (L, L, L)), x, np.zeros((n, 3)),
                    np.zeros((n, 3)), np.full(n, r, dtype=np.float32))


def lattice(n: int = 1000, seed: int | None = None, d: float = 3e-3, spacing: float = 0.999,
            jitter: float = 0.004, speed: float = 0.05, spin: float = 20.0, poly: float = 0.0,
            precision: str = "fp64", walls: bool = True, gravity=(0.0, 0.0, -9.81)) -> Workload:
    """Dense block on a jittered cubic lattice with spacing `spacing`*d (slightly below
    one diameter, so most neighbours touch), random velocities (|v| ~ speed) and spins.
    `poly` > 0 draws radii uniformly in [r(1-poly), r] instead of a single size."""
    rng = np.random.Generator(np.random.PCG64(seed_for(1) if seed is None else seed))
    r = 0.5 * d
    a = spacing * d
    m = int(math.ceil(n ** (1.0 / 3.0)))
    idx = np.arange(n)
    ijk = np.stack([idx % m, (idx // m) % m, idx // (m * m)], axis=1).astype(float)
    x = (ijk + 0.5) * a + r + rng.uniform(-jitter, jitter, (n, 3)) * d
    L = m * a + 2 * r + 2 * jitter * d
    v = rng.normal(0.0, speed, (n, 3))
    w = rng.normal(0.0, spin, (n, 3))
    if poly > 0:
        rad = rng.uniform(r * (1.0 - poly), r, n).astype(np.float32)
    else:
        rad = np.full(n, r, dtype=np.float32)
    cfg = _base_cfg(domain_lo=(0.0, 0.0, 0.0), domain_hi=(L, L, L), gravity=tuple(gravity),
                    precision=precision)
    wl = box_walls((0, 0, 0), (L, L, L)) if walls else []
    return Workload("lattice", cfg, wl, x, v, w, rad)


def _fcc(a: float, lo, hi):
    """FCC lattice points with nearest-neighbour distance a inside the box [lo, hi]."""
    c = a * math.sqrt(2.0)
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    n = np.ceil((hi - lo) / c).astype(int) + 1
    g = np.stack(np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij"),
                 axis=-1).reshape(-1, 3).astype(float)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts = (g[:, None, :] + basis[None, :, :]).reshape(-1, 3) * c + lo
    keep = np.all((pts >= lo) & (pts <= hi), axis=1)
    return pts[keep]


def drum(n: int = 200_000, seed: int | None = None, rmin: float = 1.5e-3, rmax: float = 2.5e-3,
         omega: float = 1.0, precision: str = "fp64", fill_scale: float | None = None,
         mu_slide: float = 0.3, restitution: float = 0.9, spacing: float = 1.02,
         spin: float = 0.0) -> Workload:
    """Rotating drum, horizontal axis along y, polydisperse spheres on an FCC lattice.

    The drum keeps the aspect L/R = 0.1/0.12 of the rotating-drum case and is sized so
    that the spheres fill half of it at a packing fraction of 0.6 (for 200k spheres of
    r in U[1.5, 2.5] mm this gives R = 0.2085 m, L = 0.1738 m)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(2) if seed is None else seed))
    rad = rng.uniform(rmin, rmax, n).astype(np.float32)
    solid = float(np.sum(4.0 / 3.0 * math.pi * rad.astype(np.float64) ** 3))
    aspect = 0.1 / 0.12
    # half full at packing fraction 0.6:  pi R^2 L / 2 * 0.6 = solid, L = aspect R
    R = (solid / (0.3 * math.pi * aspect)) ** (1.0 / 3.0)
    if fill_scale is not None:
        R *= fill_scale
    dmax = 2.0 * rmax
    a = spacing * dmax
    while True:
        # small drums lose a larger share of lattice sites to the wall margins: grow the
        # drum (by 1 % steps) only when the lattice would not hold all the spheres
        L = aspect * R
        pts = _fcc(a, (-R, 0.0, -R), (R, L, R))
        rho = np.hypot(pts[:, 0], pts[:, 2])
        inside = (rho < R - 0.55 * dmax) & (pts[:, 1] > 0.55 * dmax) & (pts[:, 1] < L - 0.55 * dmax)
        pts = pts[inside]
        if len(pts) >= n:
            break
        R *= 1.01
    pts = pts[np.argsort(pts[:, 2], kind="stable")][:n]     # lowest lattice sites first
    x = pts + rng.uniform(-0.01, 0.01, pts.shape) * dmax
    axis = (0.0, 1.0, 0.0)
    walls = [cylinder((0, 0, 0), axis, R, omega=omega, rot_origin=(0, 0, 0), rot_axis=axis),
             plane((0, 0, 0), (0, 1, 0), omega=omega, rot_origin=(0, 0, 0), rot_axis=axis),
             plane((0, L, 0), (0, -1, 0), omega=omega, rot_origin=(0, 0, 0), rot_axis=axis)]
    mat = material(restitution=restitution, mu_slide=mu_slide)
    cfg = _base_cfg(domain_lo=(-R, 0.0, -R), domain_hi=(R, L, R), dt=5e-6, particle=mat,
                    wall=dict(mat), precision=precision)
    cfg["drum_radius"] = R
    cfg["drum_length"] = L
    w = rng.normal(0.0, spin, (n, 3)) if spin > 0 else np.zeros((n, 3))
    return Workload("drum", cfg, walls, x, np.zeros((n, 3)), w, rad)


def silo(n: int = 4_300_000, seed: int | None = None, d: float = 5e-3, R: float = 0.5,
         orifice: float = 0.05, height: float = 1.0, t_open: float = 1e300,
         precision: str = "mixed", spacing: float = 1.1, jitter: float = 0.025,
         z_sink: float = -0.1) -> Workload:
    """Flat-bottomed cylindrical silo: cylinder wall, annular bottom with a central
    orifice, a floating plug over the orifice until t_open; simple cubic fill at
    `spacing` d with jitter <= `jitter` d (1.1 and 0.025: a loose fill that falls and
    packs; 0.995 and 0.002: a packed bed in which every sphere touches its lattice
    neighbours).  Search with a skin of 0.5 d (r_c = 1.5 d), rebuilt when a displacement
    exceeds 0.25 d; particles are removed below z_sink (default 0.1 m below the orifice)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(3) if seed is None else seed))
    r = 0.5 * d
    a = spacing * d
    m = int(math.floor((2 * (R - r)) / a))
    coords = (np.arange(m) - (m - 1) / 2.0) * a
    X, Y = np.meshgrid(coords, coords, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    keep = np.hypot(X, Y) < R - r - max(0.05 * d, 2 * jitter * d)
    X, Y = X[keep], Y[keep]
    per_layer = len(X)
    layers = int(math.ceil(n / per_layer))
    Z = r + max(0.05 * d, 2 * jitter * d) + np.arange(layers) * a
    x = np.empty((layers * per_layer, 3))
    x[:, 0] = np.tile(X, layers)
    x[:, 1] = np.tile(Y, layers)
    x[:, 2] = np.repeat(Z, per_layer)
    x = x[:n] + rng.uniform(-jitter, jitter, (n, 3)) * d
    top = max(height, float(x[:, 2].max()) + 2 * d)
    walls = [cylinder((0, 0, 0), (0, 0, 1), R),
             annulus((0, 0, 0), (0, 0, 1), R, orifice),
             plane((0, 0, 0), (0, 0, 1), t_off=t_open)]
    mat = material(mu_slide=0.5, mu_roll=0.1)
    cfg = _base_cfg(domain_lo=(-R, -R, z_sink - d), domain_hi=(R, R, top), dt=1e-5,
                    particle=mat, wall=dict(mat), skin=0.5 * d, z_sink=z_sink,
                    precision=precision)
    return Workload("silo", cfg, walls, x, np.zeros((n, 3)), np.zeros((n, 3)),
                    np.full(n, r, dtype=np.float32))


def batched_drums(n_instances: int = 512, seed: int | None = None, n_lo: int = 500, n_hi: int = 20_000,
                  rmin: float = 1e-3, rmax: float = 3e-3, precision: str = "mixed", dt: float = 5e-6,
                  slots=None) -> Workload:
    """Many independent rotating drums in one batch (one context, cfg["instances"]).

    Instance k is seeded with ``seed_for(4, k)`` (or ``seed + k``): particle count
    log-uniform in [n_lo, n_hi], radii uniform in [rmin, rmax], drum speed uniform in
    [0.5, 3] rad/s, sliding friction uniform in [0.2, 0.6], restitution uniform in
    [0.7, 0.95]; the other material constants are those of the single drum.  Each drum has
    the single drum's aspect L/R = 0.1/0.12 and is sized for half fill at a packing
    fraction of 0.6 (the paper does not size them), enlarged until an FCC lattice at the
    largest diameter holds all its spheres (radii spread over a factor 3 need about 8 %
    more radius), filled from the bottom, axis along y, and placed in its own slot of a regular 3D grid of equal slots
    centred on the origin, one search radius apart; every drum rotates about its own axis.
    The drums' particles are concatenated in instance order."""
    xs, rs, insts = [], [], []
    specs = []
    for k in range(n_instances):
        rng = np.random.Generator(np.random.PCG64((seed_for(4, k) if seed is None else seed + k)))
        nk = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        rad = rng.uniform(rmin, rmax, nk).astype(np.float32)
        omega = float(rng.uniform(0.5, 3.0))
        mu = float(rng.uniform(0.2, 0.6))
        e = float(rng.uniform(0.7, 0.95))
        solid = float(np.sum(4.0 / 3.0 * math.pi * rad.astype(np.float64) ** 3))
        aspect = 0.1 / 0.12
        R = (solid / (0.3 * math.pi * aspect)) ** (1.0 / 3.0)
        # an FCC lattice at the largest diameter holds fewer spheres than a half-full drum of
        # this size when the radii spread over 1-3 mm: grow the drum until it holds them all
        dk = 2.0 * float(rad.max())
        while len(_drum_sites(R, aspect * R, dk)) < nk:
            R *= 1.03
        specs.append((rng, nk, rad, omega, mu, e, R, aspect * R))
    dmax = 2.0 * rmax
    rc = 1.3 * dmax
    Rm = max(s[6] for s in specs)
    Lm = max(s[7] for s in specs)
    sx, sy, sz = 2 * Rm + 2 * rc, Lm + 2 * rc, 2 * Rm + 2 * rc
    if slots is None:
        m = int(math.ceil(n_instances ** (1.0 / 3.0) - 1e-9))
        slots = (m, m, int(math.ceil(n_instances / (m * m))))
    lo = np.array([-0.5 * slots[0] * sx, -0.5 * slots[1] * sy, -0.5 * slots[2] * sz])
    first = 0
    for k, (rng, nk, rad, omega, mu, e, R, L) in enumerate(specs):
        ix, iy, iz = k % slots[0], (k // slots[0]) % slots[1], k // (slots[0] * slots[1])
        # drum axis through (cx, y0 .. y0 + L, cz)
        cx = lo[0] + (ix + 0.5) * sx
        y0 = lo[1] + iy * sy + rc
        cz = lo[2] + (iz + 0.5) * sz
        dk = 2.0 * float(rad.max())
        pts = _drum_sites(R, L, dk)
        pts = pts[np.argsort(pts[:, 2], kind="stable")][:nk]
        x = pts + rng.uniform(-0.01, 0.01, pts.shape) * dk + np.array([cx, y0, cz])
        axis = (0.0, 1.0, 0.0)
        c = (cx, 0.0, cz)
        walls = [cylinder(c, axis, R, omega=omega, rot_origin=c, rot_axis=axis),
                 plane((cx, y0, cz), (0, 1, 0), omega=omega, rot_origin=c, rot_axis=axis),
                 plane((cx, y0 + L, cz), (0, -1, 0), omega=omega, rot_origin=c, rot_axis=axis)]
        mat = material(restitution=e, mu_slide=mu)
        insts.append(dict(first=first, particle=mat, wall=dict(mat), walls=walls, n=nk, omega=omega,
                          radius=R, length=L, center=c, y0=y0))
        xs.append(x)
        rs.append(rad)
        first += nk
    x = np.concatenate(xs)
    rad = np.concatenate(rs)
    n = len(rad)
    hi = -lo
    cfg = _base_cfg(domain_lo=tuple(lo), domain_hi=tuple(hi), dt=dt, particle=insts[0]["particle"],
                    wall=dict(insts[0]["particle"]), precision=precision)
    cfg["instances"] = insts
    cfg["n_instances"] = n_instances
    return Workload("batched-drums", cfg, [], x, np.zeros((n, 3)), np.zeros((n, 3)), rad)


def _drum_sites(R, L, dk):
    """FCC sites (spacing 1.02 dk) inside a drum of radius R and length L along y, kept
    0.55 dk from the walls."""
    pts = _fcc(1.02 * dk, (-R, 0.0, -R), (R, L, R))
    rho = np.hypot(pts[:, 0], pts[:, 2])
    inside = (rho < R - 0.55 * dk) & (pts[:, 1] > 0.55 * dk) & (pts[:, 1] < L - 0.55 * dk)
    return pts[inside]


def instance_workload(batch: Workload, k: int) -> Workload:
    """Instance k of a batch as a single system (same coordinates, walls and materials), for
    comparing the batch with plain one-system runs and with the oracle."""
    I = batch.cfg["instances"][k]
    lo, hi = I["first"], I["first"] + I["n"]
    cx, y0, cz = I["center"][0], I["y0"], I["center"][2]
    R, L = I["radius"], I["length"]
    pad = 1.3 * 2.0 * float(batch.radius.max())
    cfg = dict(batch.cfg)
    cfg.pop("instances")
    cfg.pop("n_instances")
    cfg.update(particle=I["particle"], wall=I["wall"],
               domain_lo=(cx - R - pad, y0 - pad, cz - R - pad), domain_hi=(cx + R + pad, y0 + L + pad, cz + R + pad))
    return Workload(f"drum-{k}", cfg, list(I["walls"]), batch.x[lo:hi].copy(), batch.v[lo:hi].copy(),
                    batch.w[lo:hi].copy(), batch.radius[lo:hi].copy())


def dam_break_depth(n: int, d: float = 1e-3) -> float:
    """Depth of the dam-break box for n spheres: 0.01 m per 160,000 spheres, the paper's
    weak-scaling rule (Table weak_scaling), and at least four diameters."""
    return max(0.01 * n / 160_000, 4.0 * d)


def dam_break(n: int = 160_000, seed: int | None = None, d: float = 1e-3, length: float = 0.2,
              height: float = 0.3, t_dam: float = 0.05, precision: str = "mixed", spacing: float = 1.05,
              jitter: float = 0.02, depth: float | None = None) -> Workload:
    """Dam break, the paper's weak-scaling case: monodisperse spheres fill the left half of
    a box (x in [0, length], z up to height) behind a floating wall (the dam, at
    x = length / 2) that disappears at t_dam; the depth (y) grows with the particle count,
    0.01 m per 160,000 spheres, as in the paper's weak-scaling table.  The paper gives
    neither the sphere size nor the box length and height: d = 1 mm and a 0.2 m x 0.2 m
    cross-section hold the 160,000 spheres of a 0.01 m slab about 0.14 m high.  Filled on a
    jittered cubic lattice at `spacing` d from the floor; material of the 1,000-sphere
    cube; dt = 4e-6 s (about a tenth of the Rayleigh time of a 1 mm sphere)."""
    rng = np.random.Generator(np.random.PCG64(seed_for(6) if seed is None else seed))
    if depth is None:
        depth = dam_break_depth(n, d)
    r = 0.5 * d
    a = spacing * d
    half = 0.5 * length
    nx = int(math.floor((half - d) / a))
    ny = max(1, int(math.floor((depth - d) / a)))
    per_layer = nx * ny
    layers = int(math.ceil(n / per_layer))
    X, Y = np.meshgrid(r + 0.5 * (d - a) + a * (np.arange(nx) + 0.5), r + 0.5 * (d - a) + a * (np.arange(ny) + 0.5),
                       indexing="ij")
    x = np.empty((layers * per_layer, 3))
    x[:, 0] = np.tile(X.ravel(), layers)
    x[:, 1] = np.tile(Y.ravel(), layers)
    x[:, 2] = np.repeat(r + 0.5 * (a - d) + np.arange(layers) * a, per_layer)
    if x[:n, 2].max() > height - r:
        raise RuntimeError("dam break: the box is too low for this many spheres")
    x = x[:n] + rng.uniform(-jitter, jitter, (n, 3)) * d
    walls = box_walls((0.0, 0.0, 0.0), (length, depth, height))
    walls.append(plane((half, 0.0, 0.0), (-1.0, 0.0, 0.0), t_off=t_dam))   # the dam
    cfg = _base_cfg(domain_lo=(0.0, 0.0, 0.0), domain_hi=(length, depth, height), dt=4e-6,
                    precision=precision)
    return Workload("dam-break", cfg, walls, x, np.zeros((n, 3)), np.zeros((n, 3)),
                    np.full(n, r, dtype=np.float32))
