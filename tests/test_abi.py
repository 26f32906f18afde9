"""The C ABI library builds, loads, exports every declared entry point, and its ctypes
mirror has the same struct layout as include/dem.h.  No GPU is needed: only host-side
entry points (workspace sizing, argument validation, status strings) are called."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2106_09576_gb300 import build as B
from paper_2106_09576_gb300 import dem as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dem.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load_library()


def declared_functions(header=HEADER, prefix="dem_"):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(" + prefix + r"[a-z0-9_]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dem_[a-z_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)
    assert sorted(D.EXPORTED) == names
    # the surrogate's entry points (include/surrogate.h)
    from paper_2106_09576_gb300 import surrogate as SG
    snames = declared_functions(os.path.join(ROOT, "include", "surrogate.h"), "surr_")
    assert len(snames) >= 12 and sorted(SG.SURR_FUNCS) == snames
    sexported = set(re.findall(r" T (surr_[a-z0-9_]+)", out))
    assert not [n for n in snames if n not in sexported]


LAYOUT_PROG = r"""
#include <stdio.h>
#include <stddef.h>
#include "dem.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("dem_config %zu\ndem_wall %zu\ndem_stats %zu\ndem_material %zu\ndem_instance %zu\n",
         sizeof(dem_config), sizeof(dem_wall), sizeof(dem_stats), sizeof(dem_material), sizeof(dem_instance));
  F(dem_config, radius_max) F(dem_config, gravity) F(dem_config, rebuild_every)
  F(dem_config, n_instances) F(dem_config, domain_lo) F(dem_config, z_sink) F(dem_config, max_overlap_ratio)
  F(dem_config, step_block)
  F(dem_instance, particle) F(dem_instance, wall) F(dem_instance, n_walls) F(dem_instance, walls)
  F(dem_wall, point) F(dem_wall, radius) F(dem_wall, omega) F(dem_wall, t_off)
  F(dem_stats, time) F(dem_stats, status_bits) F(dem_stats, required_workspace)
  return 0;
}
"""


def test_ctypes_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_PROG)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(got["dem_config"]) == C.sizeof(D.Config)
    assert int(got["dem_wall"]) == C.sizeof(D.Wall)
    assert int(got["dem_stats"]) == C.sizeof(D.Stats)
    assert int(got["dem_material"]) == C.sizeof(D.Material)
    assert int(got["dem_instance"]) == C.sizeof(D.Instance)
    for key, val in got.items():
        if "." not in key:
            continue
        T, f = key.split(".")
        cls = {"dem_config": D.Config, "dem_wall": D.Wall, "dem_stats": D.Stats, "dem_instance": D.Instance}[T]
        assert getattr(cls, f).offset == int(val), key


def cfg_dict(**kw):
    m = dict(young=1e7, poisson=0.3, restitution=0.9, mu_slide=0.3, mu_roll=0.1)
    c = dict(density=2500.0, particle=m, wall=dict(m), gravity=(0, 0, -9.81), dt=1e-5,
             domain_lo=(0, 0, 0), domain_hi=(0.1, 0.1, 0.1))
    c.update(kw)
    return c


def test_workspace_bytes_and_validation(lib):
    size = C.c_size_t(0)
    cfg = D.make_config(cfg_dict(), 1000, 1.5e-3)
    assert lib.dem_workspace_bytes(C.byref(cfg), C.byref(size)) == 0
    assert size.value > 1000 * 100
    big = D.make_config(cfg_dict(), 4_300_000, 2.5e-3)
    s2 = C.c_size_t(0)
    assert lib.dem_workspace_bytes(C.byref(big), C.byref(s2)) == 0
    assert s2.value > size.value
    for bad in (dict(dt=0.0), dict(density=-1.0), dict(domain_hi=(0, 0.1, 0.1))):
        c = D.make_config(cfg_dict(**bad), 1000, 1.5e-3)
        assert lib.dem_workspace_bytes(C.byref(c), C.byref(size)) == 1
    c = D.make_config(cfg_dict(), 0, 1.5e-3)
    assert lib.dem_workspace_bytes(C.byref(c), C.byref(size)) == 1
    c = D.make_config(cfg_dict(), 10, 1.5e-3, precision=3)
    assert lib.dem_workspace_bytes(C.byref(c), C.byref(size)) == 1
    bad_mat = cfg_dict()
    bad_mat["particle"] = dict(bad_mat["particle"], restitution=0.0)
    c = D.make_config(bad_mat, 10, 1.5e-3)
    assert lib.dem_workspace_bytes(C.byref(c), C.byref(size)) == 1
    # a batch needs room for its instance tables; bad batch and block settings are rejected
    c = D.make_config(cfg_dict(n_instances=4), 1000, 1.5e-3)
    s3 = C.c_size_t(0)
    assert lib.dem_workspace_bytes(C.byref(c), C.byref(s3)) == 0 and s3.value > size.value
    for bad in (dict(n_instances=-1), dict(n_instances=2000), dict(step_block=48), dict(pair_eval=2),
                dict(pair_eval=-1)):
        c = D.make_config(cfg_dict(**bad), 1000, 1.5e-3)
        assert lib.dem_workspace_bytes(C.byref(c), C.byref(size)) == 1
    # one evaluation per pair needs its records and owned-slot entries (mixed contexts only)
    sizes = {}
    for prec in ("mixed", "fp64"):
        for pe in ("once", "both"):
            c = D.make_config(cfg_dict(pair_eval=pe), 1000, 1.5e-3, precision=prec)
            sz = C.c_size_t(0)
            assert lib.dem_workspace_bytes(C.byref(c), C.byref(sz)) == 0
            sizes[prec, pe] = sz.value
    assert sizes["mixed", "once"] > sizes["mixed", "both"] > sizes["fp64", "once"] == sizes["fp64", "both"]


def test_create_rejects_null_arguments_without_touching_the_device(lib):
    cfg = D.make_config(cfg_dict(), 10, 1.5e-3)
    h = C.c_void_p()
    assert lib.dem_create(C.byref(cfg), None, None, None, None, None, 0, None, C.byref(h)) == 1
    assert lib.dem_step(None, 1) == 1
    assert lib.dem_get_stats(None, None) == 1
    assert lib.dem_set_instances(None, None, 0) == 1


def test_status_strings(lib):
    for code in range(8):
        assert lib.dem_status_string(code)
    assert b"unknown" in lib.dem_status_string(99)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2106_09576_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "dem_oracle" not in text, f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no silent fallback: without the compiled library the binding refuses to run
    monkeypatch.setattr(B, "LIB", str(tmp_path / "absent" / "libdem_gb300.so"))
    monkeypatch.setattr(D, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        D.load_library(build_if_missing=False)


def test_no_cpu_path_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import workloads
    wl = workloads.lattice(n=64, seed=1)
    with pytest.raises(RuntimeError):
        D.DEM(wl.cfg, wl.x, wl.v, wl.w, wl.radius, wl.walls, precision="fp64")


def test_history_arrays_are_checked_against_the_shapes_the_call_reads():
    import numpy as np
    pairs, dtp, dtw = D.history_arrays([[0, 1], [2, 3]], np.zeros(6), np.zeros((4, 2, 3)), 4, 2)
    assert pairs.dtype == np.int32 and pairs.shape == (2, 2) and dtp.shape == (2, 3) and dtw.shape == (4, 2, 3)
    assert D.history_arrays(np.zeros((0, 2)), np.zeros((0, 3)), None, 4, 0)[2] is None
    with pytest.raises(ValueError):
        D.history_arrays([[0, 1], [2, 3]], np.zeros((1, 3)), None, 4, 0)      # too few values
    with pytest.raises(ValueError):
        D.history_arrays([[0, 4]], np.zeros((1, 3)), None, 4, 0)              # index out of range
    with pytest.raises(ValueError):
        D.history_arrays([[0, 1]], np.zeros((1, 3)), np.zeros((4, 3)), 4, 1)  # wall array shape


def test_batch_instances_marshal_as_the_workload_states():
    import workloads
    wl = workloads.batched_drums(n_instances=8, n_lo=500, n_hi=600)
    inst = wl.cfg["instances"]
    arr = D.make_instances(inst)
    assert len(arr) == 8
    for k, I in enumerate(inst):
        a = arr[k]
        assert a.first == I["first"] and a.n_walls == 3
        assert a.particle.mu_slide == I["particle"]["mu_slide"] and a.wall.restitution == I["wall"]["restitution"]
        assert a.walls[0].kind == 1 and a.walls[0].radius == I["radius"]
        assert tuple(a.walls[0].point) == tuple(map(float, I["center"])) and a.walls[0].omega == I["omega"]
        assert a.walls[1].kind == 0 and a.walls[2].kind == 0
    assert [a.first for a in arr] == sorted(a.first for a in arr)
    too_many = [dict(inst[0], walls=inst[0]["walls"] * 2)]
    with pytest.raises(ValueError):
        D.make_instances(too_many)


def test_every_cuda_source_is_built_for_sm_103a():
    csrc = os.path.join(ROOT, "paper_2106_09576_gb300", "csrc")
    assert {f for f in os.listdir(csrc) if f.endswith(".cu")} == set(B.SOURCES)
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_static_pair_search_checks_its_tensors_before_any_call():
    """find_pairs_static refuses tensors the C call would misread (wrong dtype, shape,
    strides or device) before it touches the library or a device."""
    import torch

    from paper_2106_09576_gb300.dem import find_pairs_static
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    for bad in (torch.zeros((10, 3), dtype=torch.float64),            # host tensor
                torch.zeros((10, 3), dtype=torch.float32),
                torch.zeros((3, 10), dtype=torch.float64).t(),         # strided
                torch.zeros((10, 4), dtype=torch.float64)):
        with pytest.raises(ValueError):
            find_pairs_static(bad, 0.1, lo, hi)


def test_static_pair_limits_in_the_header():
    """The static search's limits: the pair total that the 32-bit offsets can hold, and a
    scratch layout that fits the advertised particle and cell limits (the library's own
    static_assert checks the latter at build time)."""
    txt = open(os.path.join(ROOT, "include", "dem.h")).read()
    vals = dict(re.findall(r"#define (DEM_STATIC_MAX_\w+) (\d+)", txt))
    assert int(vals["DEM_STATIC_MAX_PAIRS"]) == 2 ** 31 - 1
    assert int(vals["DEM_STATIC_MAX_PARTICLES"]) == 262144 and int(vals["DEM_STATIC_MAX_CELLS"]) == 524288
