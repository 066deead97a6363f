"""Host-side check of the tile index map every kernel uses (tile_base / tile_z of the library's
internal header, compiled for the host with nvcc; no GPU): for a layout with tile bits
[0, c) and [h, h + w), the tiles b = 0 .. 2^(n - c - w) - 1 and positions j = 0 .. 2^(c + w) - 1
visit every index of a 2^n vector exactly once, tile b's own bits are [0, c) and [h, h + w),
and a flip of a tile bit stays inside the tile (j -> j ^ bit maps z -> z ^ index bit)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "aqc_internal.h"
using namespace aqc;

int main(int argc, char** argv) {
  const int n = atoi(argv[1]);
  Layout L;
  L.c = atoi(argv[2]);
  L.h = atoi(argv[3]);
  L.w = atoi(argv[4]);
  L.t = L.c + L.w;
  L.cb = 0;
  const uint64_t N = 1ull << n, T = 1ull << L.t, ntiles = N >> L.t;
  std::vector<unsigned char> seen(N, 0);
  const uint32_t in_tile = ((1u << L.c) - 1u) | (L.w ? (((1u << L.w) - 1u) << L.h) : 0u);
  for (uint64_t b = 0; b < ntiles; b++) {
    const uint32_t zb = tile_base(L, (uint32_t)b);
    if (zb & in_tile) { printf("base %llu has tile bits\n", (unsigned long long)b); return 1; }
    for (uint64_t j = 0; j < T; j++) {
      const uint32_t z = tile_z(L, (uint32_t)j, zb);
      if (z >= N || seen[z]) { printf("tile %llu pos %llu -> %u twice or out of range\n", (unsigned long long)b,
                                      (unsigned long long)j, z); return 1; }
      seen[z] = 1;
      for (int k = 0; k < L.t; k++) {  // flip of tile bit k = flip of one index bit
        const uint32_t zk = tile_z(L, (uint32_t)(j ^ (1ull << k)), zb);
        const uint32_t bit = k < L.c ? (1u << k) : (1u << (L.h + k - L.c));
        if ((z ^ zk) != bit) { printf("flip of tile bit %d is not one index bit\n", k); return 1; }
      }
    }
  }
  printf("ok\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("tilemap")
    src = d / "tilemap.cu"
    src.write_text(HARNESS)
    exe = d / "tilemap"
    inc = os.path.join(ROOT, "paper_1311_3938_gb300", "csrc")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-I", inc, "-o", str(exe), str(src)])
    return str(exe)


@pytest.mark.parametrize(
    "n,c,h,w",
    [
        (13, 13, 13, 0),  # one contiguous layout [0, 13)
        (20, 13, 13, 0),  # layout 0 of a larger state
        (20, 5, 13, 7),   # a strided layout: 256-byte chunks of complex64, bits [13, 20)
        (22, 5, 13, 8),
        (22, 4, 14, 8),   # complex128 chunk width
        (22, 6, 16, 6),   # a widened last layout
        (21, 8, 17, 4),   # the 1 KiB-chunk last layout shape
        (12, 2, 5, 4),
    ],
)
def test_tiles_partition_the_index_space(harness, n, c, h, w):
    out = subprocess.run([harness, str(n), str(c), str(h), str(w)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
