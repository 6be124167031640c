"""Host-side check of the face sweeps' launch geometry (no GPU): for every kernel family
(forward/record tiles and the statistics/adjoint tiles), every axis, K, number of
variables, periodic (wrapped) and transmissive lines and ragged grid sizes, the grid and
block that face_grid() returns, walked with the face kernel's own thread-to-face mapping
(face f = f0 + row, x column x0 + lane; active when f < n_a (wrapped) or f <= n_a, and the
column inside the grid), cover every face of every line exactly once, and the block size
is the tile's thread count (FaceTile<..>::THREADS).  The program is compiled with nvcc
and run on the host."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "tenom_internal.h"
using namespace tenom;

template <int NV, int K, int AXIS, bool FWDT>
static int check(const int* n, bool wrapped) {
  using T = FaceTile<NV, K, AXIS, FWDT>;
  dim3 grid, block;
  face_grid(NV, AXIS, n, K, &grid, &block, wrapped, FWDT);
  if ((int)block.x != T::THREADS) return 1;
  const int na = n[AXIS];
  const int nf = na + 1;
  const long long lines = (long long)n[0] * n[1] * n[2] / na;
  std::vector<int> hits((size_t)(lines * nf), 0);
  for (unsigned bx = 0; bx < grid.x; ++bx)
    for (unsigned by = 0; by < grid.y; ++by)
      for (unsigned bz = 0; bz < grid.z; ++bz)
        for (int tid = 0; tid < T::THREADS; ++tid) {
          const int lane = AXIS == 0 ? 0 : tid % T::LANES;
          const int row = AXIS == 0 ? tid : tid / T::LANES;
          const int f = (int)by * T::FACES + row;
          const int x = AXIS == 0 ? 0 : (int)bx * T::LANES + lane;
          const bool active = (wrapped ? f < na : f <= na) && (AXIS == 0 || x < n[0]);
          if (!active) continue;
          long long line;
          if (AXIS == 0) line = bx;                                  /* y + ny z */
          else if (AXIS == 1) line = x + (long long)n[0] * bz;       /* x, z */
          else line = x + (long long)n[0] * bz;                      /* x, y */
          if (line >= lines) return 2;
          hits[(size_t)(line * nf + f)] += 1;
          if (wrapped && f == 0) hits[(size_t)(line * nf + na)] += 1;  /* face n_a: face 0's copy */
        }
  for (int h : hits)
    if (h != 1) return 3;
  return 0;
}

template <int NV, int K, int AXIS>
static int axis_cases(const int* n) {
  int e = 0;
  for (int w = 0; w < 2; ++w) {
    e |= check<NV, K, AXIS, true>(n, w == 1);
    e |= check<NV, K, AXIS, false>(n, false) << 2;
  }
  return e;
}

int main() {
  const int shapes[][3] = {{1, 1, 1}, {4, 1, 1}, {37, 1, 1}, {255, 1, 1}, {256, 1, 1}, {513, 1, 1},
                           {17, 23, 1}, {33, 5, 1}, {16, 300, 1}, {257, 9, 1},
                           {9, 11, 13}, {31, 18, 7}, {16, 16, 33}, {40, 3, 70}};
  int fails = 0;
  for (const auto& s : shapes) {
    const int n[3] = {s[0], s[1], s[2]};
    const int dim = (s[2] > 1) ? 3 : (s[1] > 1 ? 2 : 1);
    int e = 0;
    if (dim == 1) {
      e |= axis_cases<3, 6, 0>(n) | axis_cases<3, 8, 0>(n);
    } else if (dim == 2) {
      e |= axis_cases<4, 6, 0>(n) | axis_cases<4, 8, 0>(n) | axis_cases<4, 6, 1>(n) | axis_cases<4, 8, 1>(n);
    } else {
      e |= axis_cases<5, 6, 0>(n) | axis_cases<5, 8, 0>(n) | axis_cases<5, 6, 1>(n) | axis_cases<5, 8, 1>(n) |
           axis_cases<5, 6, 2>(n) | axis_cases<5, 8, 2>(n);
    }
    if (e) {
      std::printf("FAIL %d %d %d code %d\n", s[0], s[1], s[2], e);
      ++fails;
    }
  }
  std::printf("checked %d shapes, %d failing\n", (int)(sizeof(shapes) / sizeof(shapes[0])), fails);
  return fails ? 1 : 0;
}
"""


def test_face_grid_covers_every_face_once(tmp_path):
    from paper_2010_13289_gb300 import build as B
    src = tmp_path / "face_grid_check.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "face_grid_check"
    cmd = [B.nvcc()] + B.ARCH + ["-std=c++17", "-O1", "-I", B.INCLUDE, "-I", B.CSRC, str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("nvcc failed:\n" + r.stderr[-3000:])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "0 failing" in out.stdout
