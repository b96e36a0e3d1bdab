"""Host checks of the tensor-core operand layout and descriptors used by the contraction
kernels (BF16 for the mixed path, TF32 for the FP32 path) (no GPU): the bit packing of the
shared-memory and instruction descriptors, that the K-major core-matrix layout is a bijection onto the tile,
and that every byte one MMA instruction can address stays inside its operand buffer (under
either reading of the leading / stride byte offsets)."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_07759_gb300", "csrc")

PROBE = r'''
#include <cstdio>
#include <vector>
#include "umma.h"
using namespace tr;
int main() {
  // instruction descriptor, M = 128, N = 112
  const uint32_t id = umma_idesc_bf16_f32(128, 112);
  printf("idesc %u %u %u %u %u %u %u\n", (id >> 4) & 3, (id >> 7) & 7, (id >> 10) & 7,
         (id >> 15) & 1, (id >> 16) & 1, (id >> 17) & 63, (id >> 24) & 31);
  const uint64_t d = umma_smem_desc(0x1230, 128, 1792);
  printf("sdesc %llu %llu %llu %llu %llu\n", (unsigned long long)(d & 0x3FFF),
         (unsigned long long)((d >> 16) & 0x3FFF), (unsigned long long)((d >> 32) & 0x3FFF),
         (unsigned long long)((d >> 46) & 3), (unsigned long long)(d >> 61));
  // layout bijection and MMA extents for R x KP tiles
  int bad = 0;
  for (int kp = 16; kp <= 256; kp += 16)
    for (int R : {128, 16, 112, 160, 256}) {
      std::vector<int> seen((size_t)R * kp, 0);
      for (int r = 0; r < R; ++r)
        for (int k = 0; k < kp; ++k) {
          const uint32_t o = umma_kmajor_offset(r, k, kp);
          if (o % 2 || o >= (uint32_t)(R * kp * 2) || seen[o / 2]++) bad++;
        }
      const uint32_t sbo = (kp / 8) * 128, lbo = 128, bytes = R * kp * 2;
      for (int ks = 0; ks < kp / 16; ++ks) {
        const uint32_t start = ks * 256;
        // as intended: 16 B rows, core matrices 128 B apart along K, row groups sbo apart
        uint32_t hi = start + (R / 8 - 1) * sbo + 1 * lbo + 127;
        if (hi >= bytes) bad++;
        // with the two offsets read the other way round
        hi = start + (R / 8 - 1) * lbo + 1 * sbo + 127;
        if (hi >= bytes) bad++;
      }
    }
  printf("bad %d\n", bad);
  const uint32_t it = umma_idesc_tf32_f32(128, 96);
  printf("idesc_tf32 %u %u %u %u %u %u %u\n", (it >> 4) & 3, (it >> 7) & 7, (it >> 10) & 7,
         (it >> 15) & 1, (it >> 16) & 1, (it >> 17) & 63, (it >> 24) & 31);
  return 0;
}
'''


def test_descriptors_and_layout():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cpp")
        open(src, "w").write(PROBE)
        exe = os.path.join(d, "p")
        subprocess.run(["g++", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    idesc = [int(x) for x in out[0].split()[1:]]
    assert idesc == [1, 1, 1, 0, 0, 112 >> 3, 128 >> 4]      # F32 acc, BF16 A/B, K-major
    sdesc = [int(x) for x in out[1].split()[1:]]
    assert sdesc == [0x1230 >> 4, 128 >> 4, 1792 >> 4, 1, 0]  # version 1, no swizzle
    assert out[2] == "bad 0"
    it = [int(x) for x in out[3].split()[1:]]
    assert it == [1, 2, 2, 0, 0, 96 >> 3, 128 >> 4]          # F32 acc, TF32 A/B, K-major
