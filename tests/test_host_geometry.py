"""The CUDA path's lattice geometry (site_coords, neighbour in csrc/
common.cuh, used by every kernel) compiled as host code and checked site by
site against a brute-force neighbour table, on lattices that include the
degenerate extents 1 (a site is its own neighbour) and 2 (the +mu and -mu
neighbours coincide)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1612_07873_gb300", "csrc")

HARNESS = r"""
#include "common.cuh"
#include <cstdio>
using namespace gbmg;
int main() {
  const int shapes[4][4] = {{4, 2, 6, 3}, {1, 5, 2, 1}, {2, 2, 2, 2}, {3, 1, 1, 7}};
  long bad = 0, checked = 0;
  for (const auto& d : shapes) {
    Geom g = make_geom(d);
    for (int s = 0; s < g.vol; ++s) {
      int c[4];
      site_coords(g, s, c);
      // brute force: site order x fastest, periodic wrap
      if (c[0] + d[0] * (c[1] + d[1] * (c[2] + d[2] * c[3])) != s) ++bad;
      for (int slot = 0; slot < 9; ++slot) {
        int e[4] = {c[0], c[1], c[2], c[3]};
        if (slot > 0) {
          int mu = (slot - 1) / 2, step = (slot - 1) % 2 == 0 ? 1 : -1;
          e[mu] = ((e[mu] + step) % d[mu] + d[mu]) % d[mu];
        }
        int want = e[0] + d[0] * (e[1] + d[1] * (e[2] + d[2] * e[3]));
        if (neighbour(g, s, c, slot) != want) ++bad;
        ++checked;
      }
    }
  }
  std::printf("%ld %ld\n", checked, bad);
  return bad != 0;
}
"""


def test_cuda_geometry_matches_brute_force(tmp_path):
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not installed")
    src = tmp_path / "geom.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "geom"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = (int(v) for v in r.stdout.split())
    assert checked == 9 * (144 + 10 + 16 + 21) and bad == 0 and r.returncode == 0
