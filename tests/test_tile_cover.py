"""The emulated contraction's lower-triangle cover (csrc/tiles.cuh) on the host.

The header is compiled as plain C++ (host code) and run over every block count
up to 300: each lower 64 x 64 block pair {r, c} must be taken by exactly one
tile (by strip c at row block r, or by strip r at row block c above its
diagonal, written transposed), every row block index must lie inside the
problem, padding blocks must not be written, the per-strip form used by the
device-side list must give the same tiles as the strip-by-strip loop, and
with the column split of an H contraction whose first columns go to host
memory the tiles of the strips below the split may write only columns below
it (and the others only columns above).  The Hermitian symmetry that lets a
strip write its upper blocks transposed is the one of Eqs. (h) and (s)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1712_07206_gb300", "csrc")

HARNESS = r"""
#define __host__
#define __device__
#include <cstdio>
#include <vector>
#include "tiles.cuh"
using namespace flapw::cover;
int main() {
  for (int ncb = 1; ncb <= 300; ++ncb) {
    const int split = (int)(0.55 * ncb);
    for (int limit : {ncb, split}) {
      if (limit < 1) continue;
      std::vector<int> cnt((size_t)ncb * ncb, 0);
      long tiles = 0;
      int bad = 0;
      for_each_tile(ncb, limit, 0, ncb, [&](int j, int mask, int r0, int r1, int r2, int r3) {
        const int rb[4] = {r0, r1, r2, r3};
        ++tiles;
        for (int q = 0; q < 4; ++q) {
          if (rb[q] < 0 || rb[q] >= ncb) bad |= 1;
          if (!((mask >> q) & 1)) continue;
          const int lo = rb[q] >= j ? rb[q] : j, hi = rb[q] >= j ? j : rb[q];
          ++cnt[(size_t)lo * ncb + hi];
          const int col = hi;  // the column block the tile writes
          if (limit < ncb && ((j < limit) != (col < limit))) bad |= 2;
        }
      });
      // the per-strip form (device-side list) gives the same tiles
      long tiles2 = 0;
      for (int j = 0; j < ncb; ++j) {
        int a, e;
        segment_of(ncb, limit, j, a, e);
        if (j < a || j >= e) bad |= 4;
        tiles2 += strip_tiles(a, e, ncb, j);
      }
      if (tiles2 != tiles) bad |= 8;
      for (int r = 0; r < ncb; ++r)
        for (int c = 0; c <= r; ++c)
          if (cnt[(size_t)r * ncb + c] != 1) bad |= 16;
      if (bad) {
        printf("FAIL ncb %d limit %d code %d\n", ncb, limit, bad);
        return 1;
      }
      if (limit == ncb) printf("%d %ld\n", ncb, tiles);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def cover_counts(tmp_path_factory):
    d = tmp_path_factory.mktemp("cover")
    src = d / "cover.cpp"
    src.write_text(HARNESS)
    exe = d / "cover"
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return {int(a): int(b) for a, b in (line.split() for line in r.stdout.split("\n") if line)}


def test_every_lower_block_once_and_split_columns(cover_counts):
    assert len(cover_counts) == 300


def test_tile_counts_near_the_triangle(cover_counts):
    # four blocks per tile: at least ncb (ncb + 1) / 8 tiles; the cover pays
    # only the rounding of a few strips (N_G 3990: 63 blocks, 504 tiles against
    # 543 for 256-row tiles aligned to 256)
    for ncb, tiles in cover_counts.items():
        ideal = ncb * (ncb + 1) / 8.0
        assert tiles >= ideal
        if ncb >= 16:
            assert tiles <= 1.02 * ideal + 4, (ncb, tiles, ideal)
    assert cover_counts[63] == 504
