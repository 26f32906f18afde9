"""Host-compiled checks of device helpers that decide data layout (no GPU needed): the
cell order used by the contact-search sort must be a bijection of the grid, equal to the
plain x-fastest order when one column covers the grid, and keep neighbouring cells close."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_09576_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <vector>
#include "dem_device.cuh"
using demgb::cell_index;
int main() {
  const int grids[][3] = {{1, 1, 1}, {5, 7, 3}, {33, 17, 4}, {64, 64, 2}, {40, 31, 5}, {134, 134, 3}};
  const int shifts[] = {0, 1, 3, 4, 5, 30};
  for (auto& g : grids) {
    const int nc[3] = {g[0], g[1], g[2]};
    const int cells = nc[0] * nc[1] * nc[2];
    for (int sh : shifts) {
      std::vector<int> seen(cells, 0);
      long long far = 0, pairs = 0;
      for (int z = 0; z < nc[2]; z++)
        for (int y = 0; y < nc[1]; y++)
          for (int x = 0; x < nc[0]; x++) {
            const int c = cell_index(nc, sh, x, y, z);
            if (c < 0 || c >= cells || seen[c]++) { printf("FAIL bijection %d %d %d sh %d\n", nc[0], nc[1], nc[2], sh); return 1; }
            if (sh >= 30 && c != (z * nc[1] + y) * nc[0] + x) { printf("FAIL plain order\n"); return 1; }
            if (z + 1 < nc[2]) {
              const int d = cell_index(nc, sh, x, y, z + 1) - c;
              pairs++;
              if (d > (1 << (2 * (sh < 15 ? sh : 15)))) far++;
            }
          }
      if (sh < 15 && far) { printf("FAIL z-neighbour farther than a column layer\n"); return 1; }
    }
  }
  printf("OK\n");
  return 0;
}
"""


def test_cell_index_is_a_bijection_and_local(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "cell_index.cu"
    src.write_text(PROG)
    exe = tmp_path / "cell_index"
    r = subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout + out.stderr
