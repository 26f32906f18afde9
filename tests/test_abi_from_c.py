"""The boundary is usable from plain C: a C11 program includes both headers, links
libdem_gb300.so and calls the entry points that need no device (workspace sizing,
parameter layout, status strings, argument checks).  The same calls from C++ see the
same declarations (the headers wrap them in extern "C")."""
import os
import subprocess

import pytest

from paper_2106_09576_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

PROG = r"""
#include <stdio.h>
#include <string.h>
#include "dem.h"
#include "surrogate.h"

static dem_material steel(void) {
  dem_material m = {1e7, 0.3, 0.9, 0.3, 0.1};
  return m;
}

int main(void) {
  dem_config c;
  memset(&c, 0, sizeof c);
  c.n = 1000;
  c.density = 2500.0;
  c.radius_max = 1.5e-3;
  c.particle = steel();
  c.wall = steel();
  c.gravity[2] = -9.81;
  c.dt = 1e-5;
  c.neighbor_factor = 1.3;
  c.precision = DEM_PRECISION_MIXED;
  c.rolling_model = 1;
  for (int d = 0; d < 3; d++) c.domain_hi[d] = 0.1;
  c.z_sink = -1e300;
  size_t mixed = 0, fp64 = 0, big = 0;
  if (dem_workspace_bytes(&c, &mixed) != 0) return 10;
  c.precision = DEM_PRECISION_FP64;
  if (dem_workspace_bytes(&c, &fp64) != 0) return 11;
  c.n = 100000;
  if (dem_workspace_bytes(&c, &big) != 0) return 12;
  c.dt = 0.0;
  size_t bad = 0;
  if (dem_workspace_bytes(&c, &bad) == 0) return 13;       /* dt must be positive */
  if (dem_workspace_bytes(NULL, &bad) == 0) return 14;
  printf("ws_mixed %zu\nws_fp64 %zu\nws_big %zu\n", mixed, fp64, big);

  dem_ctx* h = NULL;
  if (dem_step(NULL, 1) == 0) return 20;                    /* no context */
  if (dem_create(&c, NULL, NULL, NULL, NULL, NULL, 0, NULL, &h) == 0) return 21;
  if (h != NULL) return 22;
  if (dem_status_string(DEM_OK) == NULL || dem_status_string(12345) == NULL) return 23;

  surr_param_layout L;
  if (surr_params(&L) != 0 || surr_params(NULL) == 0) return 30;
  printf("surr_total %lld\n", (long long)L.total);
  for (int l = 0; l < 6; l++) printf("surr_W%d %lld\nsurr_b%d %lld\n", l, (long long)L.W[l], l, (long long)L.b[l]);
  size_t sw = 0;
  if (surr_workspace_bytes(2000, 24000, &sw) != 0 || surr_workspace_bytes(-1, 0, &sw) == 0) return 31;
  printf("surr_ws %zu\n", sw);
  return 0;
}
"""


def compile_and_run(tmp_path, compiler, std, ext):
    src = tmp_path / f"user.{ext}"
    src.write_text(PROG)
    exe = tmp_path / f"user_{ext}"
    libdir = os.path.dirname(B.LIB)
    cmd = [compiler, std, "-Wall", "-Werror", "-I", INC, str(src), "-o", str(exe),
           "-L", libdir, "-Wl,-rpath," + libdir, "-l:" + os.path.basename(B.LIB)]
    subprocess.check_call(cmd)
    p = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, (p.returncode, p.stderr)
    return {k: int(v) for k, v in (line.split() for line in p.stdout.splitlines())}


@pytest.fixture(scope="module")
def built():
    B.build()


@pytest.mark.parametrize("compiler,std,ext", [("gcc", "-std=c11", "c"), ("g++", "-std=c++17", "cpp")])
def test_c_program_uses_the_boundary(built, tmp_path, compiler, std, ext):
    got = compile_and_run(tmp_path, compiler, std, ext)
    # the mixed path keeps FP32 copies and the inner list on top of the FP64 state
    assert got["ws_mixed"] > got["ws_fp64"] > 1000 * 100
    assert got["ws_big"] > 50 * got["ws_fp64"]
    # the parameter layout the header documents: W0 [16][128] b0 [128] W1 [144][128] b1 ...
    shapes = [(16, 128), (144, 128), (256, 128), (256, 128), (256, 128), (128, 8)]
    off = 0
    for l, (fan_in, fan_out) in enumerate(shapes):
        assert got[f"surr_W{l}"] == off
        off += fan_in * fan_out
        assert got[f"surr_b{l}"] == off
        off += fan_out
    assert got["surr_total"] == off
    assert got["surr_ws"] > 0


@pytest.mark.parametrize("compiler,std,ext", [("gcc", "-std=c99", "c"), ("g++", "-std=c++11", "cpp")])
def test_headers_are_strict_c99_and_cpp11(tmp_path, compiler, std, ext):
    src = tmp_path / f"hdr.{ext}"
    src.write_text('#include "dem.h"\n#include "surrogate.h"\nint main(void) { return 0; }\n')
    subprocess.check_call([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INC, str(src),
                           "-o", str(tmp_path / f"hdr_{ext}")])
