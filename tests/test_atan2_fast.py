"""CPU pin of the polynomial atan2 of the FP32 fan angles (atan2_fast in csrc/pair_math.cuh):
against the exact atan2 over random arguments of every sign and over twelve decades of ratio,
the axes and the diagonals, within 2.5 ulp and 3e-7 absolute.  Compiled for the host with g++."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2507_21686_gb300", "csrc")

PROG = r'''
#include <cmath>
#include <cstdio>
#include <random>
#include "pair_math.cuh"
int main() {
  std::mt19937_64 g(5);
  std::normal_distribution<double> n(0, 1);
  std::uniform_real_distribution<double> u(-6, 6);
  for (int i = 0; i < 400000; ++i) {
    float y = float(n(g) * std::pow(10.0, u(g))), x = float(n(g) * std::pow(10.0, u(g)));
    if (i < 16) { const float v[4] = {1.0f, -1.0f, 0.0f, 2.5f}; y = v[i % 4]; x = v[i / 4]; if (x == 0.0f && y == 0.0f) x = 1.0f; }
    std::printf("%a %a %a\n", double(y), double(x), double(sph2d::atan2_fast(y, x)));
  }
  return 0;
}
'''


def test_atan2_fast(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "a.cpp"
    src.write_text(PROG)
    exe = tmp_path / "a"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    v = np.array([float.fromhex(s) for s in out]).reshape(-1, 3)
    ref = np.arctan2(v[:, 0], v[:, 1])
    err = np.abs(v[:, 2] - ref)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    ulp[ref == 0] = np.finfo(np.float32).tiny
    assert err.max() <= 3e-7, err.max()
    assert (err / ulp).max() <= 2.5, (err / ulp).max()
    assert np.all(np.sign(v[:, 2]) == np.sign(ref))
