"""The 32-bit division by a launch-invariant divisor that the line kernels use
to decode their item index (Granlund and Montgomery's multiply-and-shift,
FastDiv in csrc/pmg_common.cuh): the header compiled for the host, every
quotient compared with integer division."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_02577_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include "pmg_common.cuh"
int main() {
  uint64_t bad = 0, checked = 0, state = 12345;
  auto next = [&]() { state = state * 6364136223846793005ull + 1442695040888963407ull; return (uint32_t)(state >> 32); };
  auto check = [&](uint32_t d, uint32_t n) {
    const pmg::FastDiv f(d);
    ++checked;
    if (f.div(n) != n / d) { if (bad < 5) std::printf("d=%u n=%u got %u\n", d, n, f.div(n)); ++bad; }
  };
  const uint32_t edge[] = {0u, 1u, 2u, 3u, 4095u, 65535u, 65536u, 0x7fffffffu, 0x80000000u, 0xfffffffeu, 0xffffffffu};
  for (uint32_t d = 1; d <= 4097; ++d) {
    for (uint32_t e : edge) check(d, e);
    for (int k = 0; k < 64; ++k) check(d, next());
    for (uint32_t q = 1; q < 5; ++q) { check(d, q * d - 1); check(d, q * d); }
  }
  const uint32_t big[] = {4099u, 65537u, 1000003u, 16777216u, 16777217u, 0x3fffffffu, 0x40000000u, 0x7ffffffeu, 0x7fffffffu};
  for (uint32_t d : big) {
    for (uint32_t e : edge) check(d, e);
    for (int k = 0; k < 100000; ++k) check(d, next());
    for (uint64_t q = 1; q * d <= 0xffffffffull; q = q * 3 + 1) { check(d, (uint32_t)(q * d - 1)); check(d, (uint32_t)(q * d)); }
  }
  std::printf("%s %llu %llu\n", bad ? "bad" : "ok", (unsigned long long)checked, (unsigned long long)bad);
  return bad ? 1 : 0;
}
"""


def test_fastdiv_matches_integer_division(tmp_path):
    gxx, nvcc = shutil.which("g++"), shutil.which("nvcc")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include") if nvcc else ""
    if not gxx or not os.path.isfile(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "fastdiv.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "fastdiv"
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", CSRC, "-I", cuda_inc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
