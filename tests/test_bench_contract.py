"""The benchmark's host side, without a GPU: the reference arm (the CPU oracle timed on a
bounded sample) prints one well-formed JSON line on rank 0 and nothing on the other ranks,
and the roofline's inputs (measured peak, recorded DRAM traffic, algorithmic bytes) are
read and computed as stated."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ARGS = ["--impl", "reference", "--n", "3000", "--steps", "2", "--warmup", "1"]


def run_bench(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + ARGS, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    p = run_bench()
    assert p.returncode == 0, p.stderr
    lines = [s for s in p.stdout.splitlines() if s.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["gpu_launches"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # 3000 spheres fit the CPU budget, so the sample is the whole system
    assert d["config"]["sample"] == 3000 and d["config"]["workload"].endswith("-3000")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert "all of it" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # the value is the sample's particle-steps over the timed steps
    assert d["value"] == pytest.approx(3000 * 2 / (d["ms_per_step"] * 2 / 1e3), rel=1e-9)


def test_reference_arm_is_silent_on_other_ranks():
    p = run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_measured_peak_is_the_copy_bandwidth():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, kind = bench.measured_hbm_peak()
    if os.path.exists(path):
        with open(path) as f:
            assert peak == float(json.load(f)["hbm_gbs"]) and kind == "measured"
    else:
        assert peak == bench.FALLBACK_HBM_GBS and kind == "fallback"


def test_recorded_traffic_scales_per_particle_and_needs_the_workload(tmp_path, monkeypatch):
    """A traffic line is used only for its kernel, its workload and the current sources'
    hash, and scales with the particle count."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# kernel workload sha bytes particles\n"
        "k_pair_mixed+k_int_mixed silo-packed abc123 4300000000 4300000\n"
        "k_step_mixed silo-packed abc123 8600000000 4300000\n"
        "k_step_mixed drum oldsha 1 1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sources_sha", lambda: "abc123")
    t = bench.recorded_traffic("k_pair_mixed+k_int_mixed", "silo-packed", 2_150_000)
    assert t == pytest.approx(2_150_000 * 1000.0)
    assert bench.recorded_traffic("k_step_mixed", "silo-packed", 4_300_000) == pytest.approx(8.6e9)
    assert bench.recorded_traffic("k_step_mixed", "drum", 1) is None          # taken on other sources
    assert bench.recorded_traffic("k_pair_mixed+k_int_mixed", "dam-break", 10) is None


def test_algorithmic_bytes_per_unit():
    st = {"n_pairs": 10, "n_touch": 3, "n_wall_touch": 2}
    assert bench.algorithmic_bytes(st, 100) == 172 * 100 + 4 * 10 + 48 * 3 + 48 * 2
    assert bench.algorithmic_bytes({"n_pairs": 0, "n_touch": 0, "n_wall_touch": 0}, 0) == 0


def test_job_rate_on_one_rank():
    # 1,000 units in 250 ms: 4,000 units per second
    assert bench.job_rate(1000.0, 250.0, 1) == pytest.approx(4000.0)


def test_clock_summary_reads_nvidia_smi_lines():
    lines = ["0, 1995, 2070, 1201.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2010, 2070, 1250.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1500, 2070, 700.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "garbage", "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    ck = bench.ClockSampler.summarize(lines)
    assert ck["sm_mhz"] == 1995.0 and ck["sm_max_mhz"] == 2070.0 and ck["samples"] == 3
    assert ck["reasons"] == ["sw_power_cap"]
    hot = bench.ClockSampler.summarize(["0, 1200, 2070, 900, 0x40, Not Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert bench.ClockSampler.summarize([])["sm_mhz"] is None


def test_recorded_pipe_counts_need_the_kernel_workload_and_sources(tmp_path, monkeypatch):
    """The FP64 roofline's instruction count is used only for its kernel, its workload and
    the current sources' hash, per particle."""
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "a.cu"
    src.write_text("kernel source")
    import hashlib
    sha = hashlib.sha256(b"kernel source").hexdigest()[:16]
    (tmp_path / "profiles" / "pipe_counts.txt").write_text(
        f"# kernel workload sha fp64 all particles\nk_step_fp64 silo-packed {sha} 600 3000 100\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pc = bench.recorded_pipe_counts("k_step_fp64", "silo-packed", ["a.cu"])
    assert pc == {"fp64_warp_inst_per_particle": 6.0, "warp_inst_per_particle": 30.0}
    assert bench.recorded_pipe_counts("k_step_fp64", "drum", ["a.cu"]) is None
    src.write_text("changed source")
    assert bench.recorded_pipe_counts("k_step_fp64", "silo-packed", ["a.cu"]) is None


def test_all_core_oracle_baseline_spreads_samples_and_sums_rates():
    """The all-core CPU baseline: well-separated sample centres, one spawned single-thread
    oracle process per core, particle-steps summed over the common wall time."""
    import workloads
    wl = workloads.lattice(n=3000, seed=4)
    c = bench._spread_centres(wl.x, 4)
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2)
    assert len(c) == 4 and d[np.triu_indices(4, 1)].min() > 0.25 * (wl.x.max(0) - wl.x.min(0)).max()
    rate, k, steps, wall = bench.oracle_rate_all_cores(wl, 0.5, 2)
    assert k == 2000 and steps >= 3 and wall > 0     # at least 2,000 spheres per process
    assert rate > 0 and np.isfinite(rate)
