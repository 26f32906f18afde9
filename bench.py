"""Benchmark of the GB300 DEM hot path: particle-steps per second and HBM roofline.

Default workload (N = 1): the 4.3M-sphere flat-bottomed cylindrical silo (d = 5 mm,
R = 0.5 m, orifice 0.05 m plugged by a floating wall), as a packed bed in which every
sphere touches its lattice neighbours, mixed precision (FP32 contact forces, FP64 state),
dt = 1e-5 s, skin 0.5 d.  Synthetic, seeded, generated on the host; no data files.

One "step" is one DEM time step of the whole system: rebuild decision, contact search
when due (cell sort, fine search, history remap), forces with history, integration.

Outputs one JSON line (rank 0).  Keys beyond the contract:
  fp64      -- the plain FP64 GPU path on the same workload (the "mixed vs FP64" of the metric)
  roofline  -- the step kernel against measured HBM bandwidth, from CUDA events around
               its launches (dem_step_profiled) and the run's own contact counts
  cpu_baseline -- the CPU oracle on a bounded sample of the same workload

--impl reference times the CPU oracle (the only reference implementation there is) on a
bounded sample of the same workload.
Multi-GPU (torchrun): each rank advances its own replica (weak scaling, no collective in
the data path); timing is barrier-bracketed and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DEM particle-steps/s on 1 GB300 (mixed vs FP64 plain), % of HBM roofline"
UNIT = "particle-steps/s"
FALLBACK_HBM_GBS = 6800.0
STEP_KERNEL_SOURCES = ["paper_2106_09576_gb300/csrc/dem_step_common.cuh", "paper_2106_09576_gb300/csrc/dem_step_mixed.cu",
                       "paper_2106_09576_gb300/csrc/dem_device.cuh"]
REBUILD_KERNELS = 14   # kernels launched by one contact search (plus one memset)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["silo", "drum", "dam", "surrogate"], default="silo",
                   help="surrogate: timings of the learned surrogate's kernels on the 200,000-sphere drum graph")
    p.add_argument("--surrogate-forward", type=int, default=0,
                   help="--workload surrogate: only run this many forward passes (for ncu)")
    p.add_argument("--n", type=int, default=None, help="override the particle count (smaller runs)")
    p.add_argument("--skin", type=float, default=None,
                   help="override the search skin, in largest diameters (analysis runs only)")
    p.add_argument("--fp64-steps", type=int, default=None)
    p.add_argument("--profile-steps", type=int, default=None)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-batched", action="store_true", help="skip the batch of 512 drums")
    p.add_argument("--batched-steps", type=int, default=10000)
    p.add_argument("--no-configs", action="store_true",
                   help="skip the other configurations' lines (cube, drum, silo discharge)")
    p.add_argument("--pair-eval", choices=["once", "both"], default="once",
                   help="mixed step: each touching pair evaluated once (its reaction handed to the "
                        "partner) or from both sides")
    return p.parse_args()


def make_workload(name, n=None, precision="mixed"):
    import workloads
    if name == "silo":
        wl = workloads.silo(n=n or 4_300_000, precision=precision, spacing=0.995, jitter=0.002)
        desc = "silo-packed"
    elif name == "dam":
        # the weak-scaling dam break at 1.6M spheres (a 0.1 m slab), packed behind the dam
        # (touching lattice), the dam gone after 500 steps
        wl = workloads.dam_break(n=n or 1_600_000, precision=precision, t_dam=0.002, spacing=0.999,
                                 jitter=0.002)
        desc = "dam-break"
    else:
        wl = workloads.drum(n=n or 200_000, precision=precision, spacing=0.999)
        desc = "drum-rotating"
    return wl, desc


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, the maximum clock and the throttle reasons seen active, from
        nvidia-smi CSV lines in the order of QUERY."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                cur, top = float(f[1]), float(f[2])
            except ValueError:
                continue
            sm.append(cur)
            smax.append(top)
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def sources_sha():
    h = hashlib.sha256()
    for rel in STEP_KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload_desc, n):
    """DRAM bytes per step (the step kernels' launches) from the committed ncu summary, if
    it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = sources_sha()
    for line in open(path):
        f = line.split()
        if len(f) >= 5 and not line.startswith("#") and f[0] == kernel and f[1] == workload_desc \
                and f[2] == sha:
            per_particle = float(f[3]) / float(f[4])
            return per_particle * n
    return None


FP64_STEP_SOURCES = ["paper_2106_09576_gb300/csrc/dem_step_common.cuh", "paper_2106_09576_gb300/csrc/dem_step_fp64.cu",
                     "paper_2106_09576_gb300/csrc/dem_device.cuh"]


def recorded_pipe_counts(kernel, workload_desc, sources):
    """FP64-pipe and all warp instructions per particle of one launch of `kernel`, from the
    committed ncu summary (profiles/pipe_counts.txt), if taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "pipe_counts.txt")
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    sha = h.hexdigest()[:16]
    for line in open(path):
        f = line.split()
        if len(f) >= 6 and not line.startswith("#") and f[0] == kernel and f[1] == workload_desc and f[2] == sha:
            n = float(f[5])
            return {"fp64_warp_inst_per_particle": float(f[3]) / n, "warp_inst_per_particle": float(f[4]) / n}
    return None


def algorithmic_bytes(st, n_active):
    """Bytes the method must move per force-and-integration launch: read x, v, w (FP64)
    and the radius (FP32), write x, v, w, read x_ref: 172 B per particle; 4 B per listed
    pair (one index), 48 B per touching pair and per particle-wall contact (FP64 tangential
    overlap read and written)."""
    return (172.0 * n_active + 4.0 * st["n_pairs"] + 48.0 * st["n_touch"] + 48.0 * st["n_wall_touch"])


def dist_setup(gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op):
    """All-reduce of one number over the ranks (NCCL on the GPUs, gloo on CPU ranks)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX) if world > 1 else x


def sum_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM) if world > 1 else x


def job_rate(units, ms, world):
    """Whole-job throughput: the units every rank processed / the slowest rank's time."""
    return sum_over_ranks(units, world) / (max_over_ranks(ms, world) / 1e3)


# ------------------------------------------------------------------ CPU oracle timing
def oracle_rate(wl, seconds, max_steps=None, warmup=0):
    """Times the CPU oracle on a bounded sample of the workload: a central vertical column
    of the silo (or a central slab of the drum) sized so the run takes about `seconds`."""
    import oracle
    import workloads
    x = wl.x
    # probe speed on a small column, then size the sample
    def column(k_target):
        r2 = x[:, 0] ** 2 + x[:, 1] ** 2 if wl.name == "silo" else x[:, 0] ** 2 + (x[:, 2] + 0.0) ** 2
        order = np.argsort(r2, kind="stable")
        return np.sort(order[:min(k_target, wl.n)])

    def sub(idx):
        return workloads.Workload("sample", dict(wl.cfg), wl.walls, x[idx], wl.v[idx], wl.w[idx], wl.radius[idx])

    probe = sub(column(4000))
    o = oracle.OracleSim(probe.cfg, probe.x, probe.v, probe.w, probe.radius, probe.walls)
    o.step(1)
    t0 = time.perf_counter()
    o.step(3)
    rate = 3 * probe.n / (time.perf_counter() - t0)
    o.close()
    steps = max_steps if max_steps is not None else 5
    k = int(max(2000, min(wl.n, rate * seconds / max(steps + warmup, 1))))
    s = sub(column(k))
    o = oracle.OracleSim(s.cfg, s.x, s.v, s.w, s.radius, s.walls)
    o.step(max(warmup, 1))                         # first search and force evaluation untimed
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    o.close()
    return s.n * steps / dt, s.n, steps, dt


def _spread_centres(x, p, seed=0):
    """p well-separated sample centres (farthest-point choice on a subsample of x)."""
    rng = np.random.default_rng(seed)
    sub = x[rng.choice(len(x), size=min(len(x), 20000), replace=False)]
    c = [sub[np.argmin(np.linalg.norm(sub - sub.mean(0), axis=1))]]
    d = np.linalg.norm(sub - c[0], axis=1)
    while len(c) < p:
        c.append(sub[int(np.argmax(d))])
        d = np.minimum(d, np.linalg.norm(sub - c[-1], axis=1))
    return np.array(c)


_BARRIER = None


def _pool_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_task(task):
    """One core's share of the all-core baseline: the oracle on its own sample, first
    search and force evaluation untimed, then `steps` steps timed from a common start."""
    cfg, walls, x, v, w, r, steps = task
    import oracle
    o = oracle.OracleSim(cfg, x, v, w, r, walls)
    o.step(1)
    _BARRIER.wait(timeout=600)
    t0 = time.monotonic()
    o.step(steps)
    t1 = time.monotonic()
    o.close()
    return len(x) * steps, t0, t1


def oracle_rate_all_cores(wl, seconds, cores):
    """The oracle on every host core at once: `cores` single-thread processes (spawned, so
    no CUDA state is inherited), each on a ball of up to n / cores (at most 200,000)
    spheres around its own well-separated centre of the workload, stepped long enough
    (from the single-thread speed) for about `seconds`; rate = all particle-steps /
    (last finish - first start)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import oracle
    import workloads
    oracle.build()
    one, _, _, _ = oracle_rate(wl, 2.0, max_steps=2)
    k = int(max(min(2000, wl.n), min(wl.n // cores, 200_000)))
    steps = int(min(200, max(3, one * seconds / k)))
    tasks = []
    for c in _spread_centres(wl.x, cores):
        idx = np.sort(np.argsort(np.linalg.norm(wl.x - c, axis=1), kind="stable")[:k])
        sw = workloads.Workload("sample", dict(wl.cfg), wl.walls, wl.x[idx], wl.v[idx], wl.w[idx], wl.radius[idx])
        tasks.append((sw.cfg, sw.walls, sw.x, sw.v, sw.w, sw.radius, steps))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    with ProcessPoolExecutor(max_workers=cores, mp_context=ctx, initializer=_pool_init,
                             initargs=(barrier,)) as ex:
        res = list(ex.map(_oracle_task, tasks))
    units = sum(u for u, _, _ in res)
    wall = max(t1 for _, _, t1 in res) - min(t0 for _, t0, _ in res)
    return units / wall, k, steps, wall


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def sample_part(k, n):
    return "all of it" if k >= n else "central column"


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, desc = make_workload(args.workload, args.n, "mixed")
    if args.skin is not None:
        wl.cfg["skin"] = args.skin * 2.0 * float(wl.radius.max())
        desc += f"-skin{args.skin:g}d"
    budget = 120.0
    rate, k, steps, dt = oracle_rate(wl, budget, max_steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "gpu_launches": 0,
        "config": {"workload": f"{desc}-{wl.n}", "sample": k, "parallelism": "single-thread CPU"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{k} spheres of the {desc} workload ({sample_part(k, wl.n)}), {steps} steps"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_batched(args, dev, world):
    """512 drums (particle counts log-uniform in 500-20,000) in one batch context, launch
    parameters picked by the autotuner, timed over --batched-steps steps from the seeded
    fill; beside it, the same drums run one system per context, timed on 16 of them spread
    over the size range and extrapolated to all 512 by particle count."""
    import torch
    import workloads
    from paper_2106_09576_gb300 import DEM
    from paper_2106_09576_gb300.autotune import autotune

    b = workloads.batched_drums(precision="mixed")
    over, table = autotune(b, device=dev)
    cfg = dict(b.cfg, **over)
    g = DEM(cfg, b.x, b.v, b.w, b.radius, b.walls, precision="mixed", device=dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    g.step(args.batched_steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_rank = e0.elapsed_time(e1)
    ms = max_over_ranks(ms_rank, world)
    st = g.stats()
    value = job_rate(b.n * args.batched_steps, ms_rank, world)
    # whole step (graph, searches included) against HBM, with the batch's own counters at
    # the last step; the working set (~1 GB) exceeds L2
    peak, peak_src = measured_hbm_peak()
    alg = algorithmic_bytes(st, st["n_active"])
    ach = alg / (ms_rank / args.batched_steps / 1e3) / 1e9
    roof = {"bound": "hbm", "unit": "GB/s", "achieved": ach, "peak": peak, "frac": ach / peak,
            "peak_source": peak_src, "kernel": "whole step (graph: k_begin, searches when due, step kernels)",
            "algorithmic_bytes_per_step": alg, "bytes_per_particle_step": alg / max(st["n_active"], 1)}
    g.close()
    del g
    torch.cuda.empty_cache()
    # plain: one context per drum, on a sample spread over the size range
    insts = b.cfg["instances"]
    order = sorted(range(len(insts)), key=lambda k: insts[k]["n"])
    sample = [order[int(round(q * (len(order) - 1)))] for q in np.linspace(0.0, 1.0, 16)]
    k_steps = min(1000, args.batched_steps)
    rates = []
    for k in sample:
        wk = workloads.instance_workload(b, k)
        wk.cfg["pair_eval"] = over["pair_eval"]          # same pair evaluation as the batch
        gk = DEM(wk.cfg, wk.x, wk.v, wk.w, wk.radius, wk.walls, precision="mixed", device=dev)
        gk.step(10)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        gk.step(k_steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        rates.append((wk.n, wk.n * k_steps / (e0.elapsed_time(e1) / 1e3)))
        gk.close()
    ns = np.array([r[0] for r in rates], float)
    rs = np.array([r[1] for r in rates], float)
    all_n = np.array([I["n"] for I in insts], float)
    est_rate = np.exp(np.interp(np.log(all_n), np.log(ns), np.log(rs)))
    plain_seconds = float(np.sum(all_n * args.batched_steps / est_rate))
    plain_value = float(all_n.sum() * args.batched_steps / plain_seconds)
    return {"workload": f"batched-drums-512 ({b.n} spheres, N log-uniform in 500-20000, r in 1-3 mm)",
            "n": b.n, "instances": len(insts), "steps": args.batched_steps, "value": value, "unit": UNIT,
            "ms_per_step": ms / args.batched_steps, "dt": b.cfg["dt"], "precision": "mixed",
            "autotune": {"chosen": over, "candidates": table}, "roofline": roof,
            "timed_from": "the seeded fill (every step of the 10,000, including the early settling and its "
                          "searches); the autotuner times 300 steps after 100 untimed ones",
            "rebuilds": st["rebuilds"], "n_touch_last_step": st["n_touch"],
            "plain": {"value": plain_value, "unit": UNIT, "method": "one context per drum, 16 drums timed over "
                      f"{k_steps} steps each, extrapolated to all 512 by particle count"},
            "speedup_vs_plain": value / plain_value,
            "state_vs_plain": "bit-identical per instance (tests/test_gpu_batch.py)"}


def timed_steps(g, steps, dev, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0 = g.stats()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    s1 = g.stats()
    ms = e0.elapsed_time(e1)
    return ms, s0, s1


def run_configs(args, dev, world):
    """C1: the 1,000-sphere cube settling in FP64 (2,000 steps); C2: the 200,000-sphere
    rotating drum, settled and turning (after 0.3 s), in mixed precision (20,000 steps) and
    FP64 (2,000 steps); C3 (ii): the
    4.3M silo discharging -- the packed bed with the orifice plug gone at t = 0, timed over
    500 steps after 3,000 steps of developing flow (searches and removals in the window)."""
    import torch
    import workloads
    from paper_2106_09576_gb300 import DEM
    stream = torch.cuda.current_stream(dev)
    out = {}

    def line(g, steps, warm, wl=None):
        g.step(warm)
        ms, s0, s1 = timed_steps(g, steps, dev, stream)
        act = 0.5 * (s0["n_active"] + s1["n_active"])
        d = {"value": job_rate(act * steps, ms, world), "unit": UNIT, "steps": steps, "warmup": warm,
             "ms_per_step": ms / steps, "searches_in_window": s1["rebuilds"] - s0["rebuilds"],
             "n_active": s1["n_active"], "n_touch": s1["n_touch"]}
        g.close()
        if wl is not None and not args.no_cpu and world == 1:
            # the oracle on the same workload (from its initial state), one core and all cores
            r1, k1, st1, _ = oracle_rate(wl, 4.0)
            cores = host_cores()
            ra, ka, sta, _ = oracle_rate_all_cores(wl, 4.0, cores) if cores > 1 else (r1, k1, st1, 0.0)
            d["oracle"] = {"single_thread": r1, "all_cores": ra, "cores": cores, "unit": UNIT,
                           "sample": f"single thread: {k1} spheres x {st1} steps; all cores: {cores} processes "
                                     f"of {ka} spheres x {sta} steps"}
        return d

    c = workloads.cube(precision="fp64")
    out["c1_cube_fp64"] = dict(workload=f"cube-{c.n}", precision="fp64",
                               **line(DEM(c.cfg, c.x, c.v, c.w, c.radius, c.walls, precision="fp64", device=dev),
                                      2000, 5, c))
    # the drum filled and turned for 0.3 s (60,000 mixed steps: a settled, rolling bed), then
    # both precisions timed from that state (positions, velocities and tangential overlaps);
    # the mixed step with each pair evaluation, the faster one reported (in a drum the ids
    # are in random order, so the owned-pair counts of a warp's particles vary from 0 to 6)
    d = workloads.drum(precision="mixed")
    gd = DEM(d.cfg, d.x, d.v, d.w, d.radius, d.walls, precision="mixed", device=dev)
    gd.step(60000)
    xs, vs, ws, _ = gd.state()
    hist = gd.history()
    gd.close()
    settled = workloads.Workload("drum", dict(d.cfg), d.walls, xs, vs, ws, d.radius)
    lines = {}
    for pe in ("once", "both"):
        cfg = dict(d.cfg)
        cfg["pair_eval"] = pe
        g = DEM(cfg, xs, vs, ws, d.radius, d.walls, precision="mixed", device=dev)
        g.set_history(*hist)
        lines[pe] = line(g, 20000, 0)
    best = min(lines, key=lambda k: lines[k]["ms_per_step"])
    out["c2_drum_mixed"] = dict(workload=f"drum-rotating-{d.n} (after 0.3 s)", precision="mixed", pair_eval=best,
                                ms_per_step_by_pair_eval={k: v["ms_per_step"] for k, v in lines.items()},
                                **lines[best])
    out["c2_drum_fp64"] = dict(workload=f"drum-rotating-{d.n} (after 0.3 s)", precision="fp64",
                               **line(DEM(settled.cfg, xs, vs, ws, d.radius, d.walls, precision="fp64", device=dev),
                                      2000, 20, settled))
    torch.cuda.empty_cache()
    sl = workloads.silo(precision="mixed", spacing=0.995, jitter=0.002, t_open=0.0)
    sl.cfg["pair_eval"] = args.pair_eval
    out["c3_silo_discharge_mixed"] = dict(
        workload=f"silo-discharge-{sl.n}", precision="mixed",
        **line(DEM(sl.cfg, sl.x, sl.v, sl.w, sl.radius, sl.walls, precision="mixed", device=dev), 500, 3000))
    # the oracle on the discharging silo is the headline's cpu_baseline workload (the bed)
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    from paper_2106_09576_gb300 import DEM

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl, desc = make_workload(args.workload, args.n, "mixed")
    if args.skin is not None:
        wl.cfg["skin"] = args.skin * 2.0 * float(wl.radius.max())
        desc += f"-skin{args.skin:g}d"
    wl.cfg["pair_eval"] = args.pair_eval
    once = args.pair_eval == "once"
    n = wl.n
    extra = {}

    # ---------------- issue rates of the arithmetic pipes (the FP64 path's ceiling)
    from paper_2106_09576_gb300.dem import pipe_rates
    pipe = pipe_rates(dev)
    extra["pipe_rates"] = {"unit": "thread instr/s", **pipe, "dfma_over_ffma": pipe["dfma"] / pipe["ffma"]}

    # ---------------- mixed precision, device-resident inputs, graph path
    g = DEM(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls, precision="mixed", device=dev)
    g.step(args.warmup)
    g.sync()
    st0 = g.stats()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    e0.record(stream)
    g.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    barrier(world)
    ms = e0.elapsed_time(e1)
    st1 = g.stats()
    ms_max = max_over_ranks(ms, world)
    active = 0.5 * (st0["n_active"] + st1["n_active"])
    value = job_rate(active * args.steps, ms, world)
    rebuilds = st1["rebuilds"] - st0["rebuilds"]
    inner_builds = st1["inner_builds"] - st0["inner_builds"]
    # k_set_remaining and k_end per dem_step call, k_begin and the step kernels per step
    # (k_pair_mixed + k_int_mixed, or k_step_mixed), and the list builds (a contact search
    # also refreshes the inner list; with one evaluation per pair a refresh is two kernels)
    per_inner = 2 if once else 1
    launches = (2 + (3 if once else 2) * args.steps + (REBUILD_KERNELS + per_inner) * rebuilds
                + per_inner * max(inner_builds - rebuilds, 0))

    # ---------------- step-kernel roofline (CUDA events around each launch)
    kp = args.profile_steps if args.profile_steps is not None else min(args.steps, 200)
    g.set_state()          # no data: makes a contact search fall due in the profiled window
    prof = g.step_profiled(kp)
    st2 = g.stats()
    kernel_ms = prof["step_kernel_ms"] / max(prof["step_launches"], 1)
    alg = algorithmic_bytes(st2, st2["n_active"])
    peak, peak_src = measured_hbm_peak()
    achieved = alg / (kernel_ms / 1e3) / 1e9
    kname = "k_pair_mixed+k_int_mixed" if once else "k_step_mixed"
    traffic = recorded_traffic(kname, desc, st2["n_active"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "peak_source": peak_src,
                "kernel_ms": kernel_ms, "algorithmic_bytes_per_launch": alg,
                "bytes_per_particle_step": alg / max(st2["n_active"], 1),
                "search_ms_avg": prof["search_ms"] / max(prof["searches"], 1), "searches": prof["searches"],
                "inner_build_ms_avg": prof["inner_ms"] / max(prof["inner_builds"], 1),
                "inner_builds": prof["inner_builds"],
                "profiled_steps": kp, "step_share_of_time": prof["step_kernel_ms"] /
                max(prof["step_kernel_ms"] + prof["search_ms"] + prof["inner_ms"], 1e-12)}
    contacts = {"n_pairs": st2["n_pairs"], "n_touch": st2["n_touch"], "n_wall_touch": st2["n_wall_touch"],
                "rebuilds_in_window": rebuilds, "inner_builds_in_window": inner_builds,
                "max_overlap_ratio": st2["max_overlap_ratio"]}

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        x_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        v_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        w_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        a_h = torch.empty((n,), dtype=torch.uint8, pin_memory=True)
        g.state((x_h, v_h, w_h, a_h))
        st_pre = g.stats()
        barrier(world)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        g.set_state(x_h, v_h, w_h, a_h)          # host -> device
        g.step(args.steps)
        g.state((x_h, v_h, w_h, a_h))            # device -> host (synchronises)
        t_e2e = time.perf_counter() - t0
        barrier(world)
        t_e2e = max_over_ranks(t_e2e, world)
        st3 = g.stats()
        e2e_val = sum_over_ranks(st3["n_active"] * args.steps, world) / t_e2e
        bytes_io = n * (3 * 3 * 8 + 1)
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": bytes_io / args.steps,
               "d2h_bytes_per_step": bytes_io / args.steps, "steps_per_call": args.steps,
               # a later window of the same run: its searches and refreshes differ from the
               # device-timed window's (set_state forces one search)
               "rebuilds_in_window": st3["rebuilds"] - st_pre["rebuilds"],
               "inner_builds_in_window": st3["inner_builds"] - st_pre["inner_builds"],
               "note": "dem_set_state(host) + dem_step(steps) + dem_get_state(host), pinned host memory"}
    g.close()
    del g
    torch.cuda.empty_cache()

    # ---------------- plain FP64 on the same workload
    if not args.no_fp64:
        kf = args.fp64_steps if args.fp64_steps is not None else max(10, min(args.steps, 100))
        gf = DEM(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls, precision="fp64", device=dev)
        gf.step(args.warmup)
        gf.sync()
        s0 = gf.stats()
        barrier(world)
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        gf.step(kf)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        fms = max_over_ranks(f0.elapsed_time(f1), world)
        s1 = gf.stats()
        fv = sum_over_ranks(0.5 * (s0["n_active"] + s1["n_active"]) * kf, world) / (fms / 1e3)
        extra["fp64"] = {"value": fv, "unit": UNIT, "steps": kf, "ms_per_step": fms / kf,
                         "mixed_speedup": value / fv}
        # the FP64 step kernel against the measured FP64 FMA rate: its FP64-pipe warp
        # instructions per launch (ncu count per particle, committed) over its CUDA-event time
        pf = gf.step_profiled(5)
        fk_ms = pf["step_kernel_ms"] / max(pf["step_launches"], 1)
        pc = recorded_pipe_counts("k_step_fp64", desc, FP64_STEP_SOURCES)
        # the pipe rates again, now that the GPU has run for seconds (the first probe can
        # catch the clock still rising): the larger of the two is the ceiling
        again = pipe_rates(dev)
        for key in ("dfma", "dadd", "ffma", "f2d"):
            pipe[key] = max(pipe[key], again[key])
        extra["pipe_rates"] = {"unit": "thread instr/s", **pipe, "dfma_over_ffma": pipe["dfma"] / pipe["ffma"]}
        peak_w = pipe["dfma"] / 32.0
        ach = None if pc is None else pc["fp64_warp_inst_per_particle"] * s1["n_active"] / (fk_ms / 1e3)
        extra["fp64"]["roofline"] = {
            "bound": "alu", "kernel": "k_step_fp64", "unit": "G FP64-pipe warp instr/s",
            "achieved": None if ach is None else ach / 1e9, "peak": peak_w / 1e9,
            "frac": None if ach is None else ach / peak_w, "kernel_ms": fk_ms,
            "peak_source": "measured (dem_pipe_rates: FP64 FMA thread rate / 32)",
            "fp64_warp_inst_per_particle": None if pc is None else pc["fp64_warp_inst_per_particle"]}
        gf.close()
        del gf
        torch.cuda.empty_cache()

    # ---------------- the other configurations, one line each
    if not args.no_configs:
        extra["configs"] = run_configs(args, dev, world)

    # ---------------- batch of 512 independent drums in one context (one launch per step)
    if not args.no_batched:
        extra["batched"] = run_batched(args, dev, world)

    # ---------------- CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if not args.no_cpu and world == 1 and rank == 0:
        rate, k, steps, dt = oracle_rate(wl, args.cpu_seconds)
        single = {"value": rate, "unit": UNIT, "cores": 1,
                  "sample": f"{k} spheres of the {desc} workload ({sample_part(k, wl.n)}), {steps} steps, "
                            f"{dt:.1f} s"}
        cores = host_cores()
        if cores > 1:
            arate, ak, asteps, adt = oracle_rate_all_cores(wl, args.cpu_seconds, cores)
            cpu = {"value": arate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{cores} single-thread oracle processes at once, each on its own ball of {ak} "
                             f"spheres of the {desc} workload, {asteps} steps, {adt:.1f} s wall, host CPU of the "
                             f"GPU box", "single_thread": single}
        else:
            cpu = dict(single, kind="oracle")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{desc}-{n}", "n": n, "precision": "mixed", "pair_eval": args.pair_eval,
                       "dt": wl.cfg["dt"],
                       "d": float(2 * wl.radius.max()), "skin": wl.cfg.get("skin", 0.0),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (state + lists + overlaps > 129 MB)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": ck,
            "contacts": contacts,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_surrogate(args):
    """Timings of the surrogate's kernels at the size of the 200,000-sphere drum (CUDA events
    after warm-up): the 128-wide product on its own, C [M][128] = A [M][K] W [K][128] with
    M = 1,228,800 and K = 144 and 256 (BF16 in, FP32 out) -- the tcgen05 kernel of the
    forward pass, the mma.sync kernel of the backward pass, and torch.matmul (cuBLAS, BF16
    out) for context; bytes = M (2 K + 4 * 128) + 2 K 128 -- and the forward and backward
    passes of the network on the radius-1.2 d graph of the drum fill (about 2.3M directed
    edges).  One JSON line."""
    import torch
    import workloads
    from paper_2106_09576_gb300 import surrogate as SG

    dev = torch.device("cuda")
    s = torch.cuda.current_stream()

    def timeit(fn, reps=10, warm=3):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    wl = workloads.drum(n=200_000, precision="mixed", spacing=0.999)
    x, v, w = (torch.tensor(a, device=dev) for a in (wl.x, wl.v, wl.w))
    r = torch.tensor(wl.radius, device=dev)
    net = SG.SurrogateNet()
    t0 = time.perf_counter()
    g = SG.Graph(x, 1.2 * 2.0 * float(wl.radius.max()), wl.cfg["domain_lo"], wl.cfg["domain_hi"])
    torch.cuda.synchronize()
    t_graph = time.perf_counter() - t0
    X, E = net.features(x, v, w, r, g, SG.drum_geometry(wl, dev))
    if args.surrogate_forward:
        for _ in range(args.surrogate_forward):
            Y = net.forward(X, E, g)
        torch.cuda.synchronize()
        print(json.dumps({"workload": "surrogate-drum-200000", "nodes": g.n, "edges": g.n_edges,
                          "forwards": args.surrogate_forward, "checksum": float(Y.abs().sum())}))
        return
    out = {"workload": "surrogate-drum-200000", "nodes": g.n, "edges": g.n_edges, "graph_s": t_graph}
    out["forward_ms"] = timeit(lambda: net.forward(X, E, g))
    Y = net.forward(X, E, g)
    dY = torch.randn_like(Y)
    out["backward_ms"] = timeit(lambda: net.backward(dY, g))
    fl = 2 * (g.n * 16 * 128 + g.n_edges * 144 * 128 + 3 * g.n * 256 * 128 + g.n * 128 * 8)
    out["forward_gflop"] = fl / 1e9
    del X, E, Y, dY, g
    M, N = 1_228_800, 128
    lib = SG.lib()
    peak, peak_src = measured_hbm_peak()
    for K in (144, 256):
        A = torch.randn(M, K, device=dev).to(torch.bfloat16)
        B = torch.randn(K, N, device=dev).to(torch.bfloat16)
        C = torch.empty(M, N, device=dev)
        byt = M * K * 2 + K * N * 2 + M * N * 4
        ref = A[:4096].float() @ B.float()
        for name, fn in (("tcgen05", lambda: lib.surr_gemm_bf16_tc(SG._p(A), SG._p(B), SG._p(C), M, K,
                                                                     SG._stream(torch, dev))),
                         ("mma_sync", lambda: lib.surr_gemm_bf16(SG._p(A), SG._p(B), SG._p(C), M, K, N,
                                                                  SG._stream(torch, dev)))):
            ms = timeit(lambda: SG._ok(name, fn()))
            err = float((C[:4096] - ref).abs().max() / ref.abs().max())
            out[f"{name}_K{K}"] = {"ms": ms, "tflops": 2 * M * N * K / ms / 1e9, "gbs": byt / ms / 1e6,
                                   "frac_of_hbm": byt / ms / 1e6 / peak, "rel_err": err}
        ms = timeit(lambda: torch.matmul(A, B))
        out[f"cublas_bf16out_K{K}"] = {"ms": ms, "gbs": (M * K * 2 + K * N * 2 + M * N * 2) / ms / 1e6}
        del A, B, C
    out["hbm_peak"] = {"value": peak, "unit": "GB/s", "source": peak_src}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "surrogate":
        run_surrogate(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
