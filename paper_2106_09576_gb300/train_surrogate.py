"""Trains the drum surrogate on DEM trajectories and compares it with plain DEM.

    python -m paper_2106_09576_gb300.train_surrogate [--trajectories 200] [--eval-steps 50000]
    python -m paper_2106_09576_gb300.train_surrogate --particles 20000 --train-settle 20000 \
        --eval-particles 200000 --settle 100000 --eval-drums 1   # trained on 20k drums, judged on 200k

1. 200 seeded DEM trajectories of small drums (the 200k drum's materials, radii and speed)
   give (state, increments over 10 steps) samples, the input velocities and spins perturbed
   by noise (0.1 of the velocity scale) so that the network learns to pull a drifting state
   back; 10 more trajectories are held out (without noise).
2. Training with the library's kernels (forward, backward, Adam).
3. On held-out drums, from a settled state: plain DEM and the surrogate with DEM fallback
   (a surrogate step is rejected when the largest overlap exceeds 2 % of the diameter or
   the kinetic energy grows by more than 20 %) each advance the same number of DEM-step
   equivalents; the dynamic angle of repose and the kinetic energy are compared, with the
   wall time per equivalent step of each.
Prints one JSON object (and writes it to --out if given).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main():
    import torch

    import workloads
    from . import surrogate as SG
    from .dem import DEM
    from .observables import angle_of_repose, kinetic_energy

    ap = argparse.ArgumentParser()
    ap.add_argument("--trajectories", type=int, default=200)
    ap.add_argument("--held-out", type=int, default=10)
    ap.add_argument("--particles", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--eval-steps", type=int, default=50000)
    ap.add_argument("--eval-drums", type=int, default=3)
    ap.add_argument("--eval-particles", type=int, default=None,
                    help="spheres of the evaluation drums (default: --particles); the network's inputs "
                         "are per sphere and per contact, so a model trained on small drums runs on large ones")
    ap.add_argument("--settle", type=int, default=20000, help="DEM steps before an evaluation rollout")
    ap.add_argument("--train-settle", type=int, default=4000, help="DEM steps before a trajectory's first sample")
    ap.add_argument("--noise-v", type=float, default=0.1, help="input velocity noise, in velocity scales")
    ap.add_argument("--noise-x", type=float, default=0.0, help="input position noise, in diameters")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--max-overlap", type=float, default=0.02, help="rollout: largest overlap, in diameters")
    ap.add_argument("--overlap-factor", type=float, default=0.0,
                    help="rollout: or this times the largest overlap of the last DEM state")
    ap.add_argument("--out", default=None)
    ap.add_argument("--save", default=None, help="write the trained parameters and output scale (.npz)")
    ap.add_argument("--load", default=None, help="skip data and training: parameters from a --save file")
    a = ap.parse_args()
    dev = torch.device("cuda")
    t0 = time.perf_counter()
    net = SG.SurrogateNet()
    if a.load:
        z = np.load(a.load)
        net.params.copy_(torch.tensor(z["params"], device=dev))
        net.out_scale.copy_(torch.tensor(z["out_scale"], device=dev))
        net.sync_bf16()
        train, hist, mse, zero, t_data, t_train = [], [], None, None, 0.0, 0.0
    else:
        train = SG.drum_trajectories(a.trajectories, a.particles, a.train_settle, 6, 60, net, noise_v=a.noise_v,
                                     noise_x=a.noise_x)
        SG.fit_output_scale(net, train)
        held = SG.drum_trajectories(a.held_out, a.particles, a.train_settle, 6, 60, net,
                                    seed0=workloads.seed_for(5, 900))
        t_data = time.perf_counter() - t0
        t0 = time.perf_counter()
        hist = SG.train(net, train, a.epochs, lr=a.lr)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        mse, zero = SG.evaluate(net, held)
        if a.save:
            np.savez(a.save, params=net.params.cpu().numpy(), out_scale=net.out_scale.cpu().numpy())

    rows = []
    n_eval = a.eval_particles or a.particles
    for k in range(a.eval_drums):
        wl = workloads.drum(n=n_eval, seed=workloads.seed_for(5, 950 + k), omega=1.0, precision="mixed",
                            spacing=0.999)
        L, dmax = wl.cfg["drum_length"], 2.0 * float(wl.radius.max())
        res = {}
        for mode in ("dem", "surrogate"):
            g = DEM(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls, precision="mixed", device=dev)
            g.step(a.settle)                                # settle and start tumbling
            torch.cuda.synchronize()
            t = time.perf_counter()
            if mode == "dem":
                g.step(a.eval_steps)
                x, v, w, act = g.state()
                fall = surr = 0
            else:
                st = {}
                (xt, vt, wt), fall, surr = SG.rollout(net, wl, g, a.eval_steps, max_overlap=a.max_overlap,
                                                      overlap_factor=a.overlap_factor, stats=st)
                x, v, w = xt.cpu().numpy(), vt.cpu().numpy(), wt.cpu().numpy()
                act = np.ones(wl.n, bool)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            res[mode] = dict(seconds=dt, us_per_equiv_step=1e6 * dt / a.eval_steps,
                             angle_deg=angle_of_repose(x, wl.radius, act, L, dmax),
                             kinetic_energy=kinetic_energy(v, w, wl.radius, wl.cfg["density"], act),
                             fallbacks=fall, surrogate_steps=surr, **(st if mode == "surrogate" else {}))
            g.close()
        rows.append(res)
    ang_err = [abs(r["surrogate"]["angle_deg"] - r["dem"]["angle_deg"]) for r in rows]
    ke_err = [abs(r["surrogate"]["kinetic_energy"] - r["dem"]["kinetic_energy"]) / max(r["dem"]["kinetic_energy"],
                                                                                       1e-30) for r in rows]
    speed = [r["dem"]["seconds"] / r["surrogate"]["seconds"] for r in rows]
    out = dict(trajectories=a.trajectories, samples=len(train), particles=a.particles, eval_particles=n_eval,
               settle_steps=a.settle, train_settle_steps=a.train_settle, epochs=a.epochs,
               noise_v=a.noise_v, noise_x=a.noise_x, lr=a.lr, max_overlap=a.max_overlap,
               overlap_factor=a.overlap_factor,
               seconds_data=t_data, seconds_train=t_train, loss_history=hist,
               held_out_mse=mse, held_out_mse_no_change=zero, eval_equiv_steps=a.eval_steps, drums=rows,
               angle_error_deg=ang_err, kinetic_energy_rel_error=ke_err, speed_vs_dem=speed)
    txt = json.dumps(out)
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt + "\n")


if __name__ == "__main__":
    main()
