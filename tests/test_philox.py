"""Philox4x32-10 (Salmon et al., SC'11) as compiled for the GPU, checked on the host against the
published known-answer vectors of the generator's reference implementation."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include "philox.cuh"
int main() {
  using namespace ffca;
  const U4 in[3] = {{0u, 0u, 0u, 0u}, {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu},
                    {0x243f6a88u, 0x85a308d3u, 0x13198a2eu, 0x03707344u}};
  const uint32_t keys[3][2] = {{0u, 0u}, {0xffffffffu, 0xffffffffu}, {0xa4093822u, 0x299f31d0u}};
  for (int i = 0; i < 3; ++i) {
    const U4 r = philox4x32_10(in[i], keys[i][0], keys[i][1]);
    printf("%08x %08x %08x %08x\n", r.x, r.y, r.z, r.w);
  }
  printf("%.9g %.9g\n", u01(0u), u01(0xffffffffu));
}
"""

KAT = ["6627e8d5 e169c58d bc57ac4c 9b00dbd8",
       "408f276d 41c83b0e a20bc7c6 6d5451fd",
       "d16cfe09 94fdcceb 5001e420 24126ea1"]


def test_philox_known_answers(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "kat.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "kat"
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "paper_2101_08563_gb300", "csrc"),
                    "-o", str(exe), str(src)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    assert out[:3] == KAT
    lo, hi = (float(v) for v in out[3].split())
    assert 0.0 < lo < 1e-7 and 1.0 - 1e-7 < hi < 1.0
