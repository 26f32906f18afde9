"""Writes silo_c3_scaled_oracle.txt: the CPU oracle's discharge of the C3-scaled silo
(seed 2106 + 3000 + 1).  Calls only oracle/ and the seeded input generator.

The silo of the 4.3M-sphere configuration scaled down for the oracle: d = 5 mm spheres of
the same material (mu_s 0.5, mu_r 0.1), a 0.05 m orifice radius, cylinder radius 0.15 m
(about 100,000 spheres), the loose simple-cubic fill of the configuration, plug removed
at t = 0.2 s, dt = 1e-5 s.  Records the number of spheres discharged every 5,000 steps
after the opening, and the packing fraction of the settled bed at the opening.

    python tests/golden/make_silo_c3_scaled.py        # about 1.5 hours on one core
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_2106_09576_gb300.observables import packing_fraction  # noqa: E402

N, R, ORIFICE, T_OPEN, D = 100_000, 0.15, 0.05, 0.2, 5e-3
SETTLE, CHUNK, MAX_STEPS = 20_000, 5_000, 200_000
SEED = workloads.seed_for(3, 1)


def silo(precision="fp64", seed=SEED):
    return workloads.silo(n=N, seed=seed, d=D, R=R, orifice=ORIFICE, height=0.5, t_open=T_OPEN,
                          precision=precision)


def main():
    oracle.build()
    wl = silo()
    o = oracle.OracleSim(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls)
    t0 = time.time()
    o.step(SETTLE)
    x, _, _, act = o.state()
    phi = packing_fraction(x, wl.radius, act, R, 0.0, D)
    rows = []
    steps = SETTLE
    while steps < MAX_STEPS:
        o.step(CHUNK)
        steps += CHUNK
        out = wl.n - o.stats()["n_active"]
        rows.append((steps, out))
        print(steps, out, f"{time.time() - t0:.0f} s", flush=True)
        if out >= 0.61 * wl.n:
            break
    with open(os.path.join(HERE, "silo_c3_scaled_oracle.txt"), "w") as f:
        f.write("# CPU oracle, C3-scaled silo (written by make_silo_c3_scaled.py): seed "
                f"{SEED}, n {N}, R {R}, orifice {ORIFICE}, t_open {T_OPEN}, dt {wl.cfg['dt']}\n")
        f.write(f"# packing fraction at the opening (probe 3 d from wall, floor and surface)\n")
        f.write(f"phi {phi!r}\n")
        f.write("# step discharged\n")
        for s, c in rows:
            f.write(f"{s} {c}\n")


if __name__ == "__main__":
    main()
