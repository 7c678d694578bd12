"""CPU pins of the compensated logarithm behind the J_-1 seed of the closed form (ff_log in
csrc/pair_math.cuh): its argument-reduction table is exactly what the committed generator
writes, every entry satisfies its definition, and the float-pair and double-pair logarithms
reach their precision against long double on the host (the same header, compiled with g++)."""
from __future__ import annotations

import math
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_21686_gb300", "csrc")


def test_table_is_the_generators_output():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_log_table.py")], capture_output=True,
                         text=True, check=True).stdout
    assert out == open(os.path.join(CSRC, "log_table.h")).read()


def _entries(name):
    txt = open(os.path.join(CSRC, "log_table.h")).read()
    body = txt.split(f"#define {name} \\")[1].split("#define")[0]
    return [tuple(float.fromhex(v.rstrip("f")) for v in m) for m in re.findall(r"\{([^,]+), ([^,]+), ([^}]+)\}", body)]


@pytest.mark.parametrize("name, eps", [("SPH2D_LOG_TABLE_F", 2.0 ** -24), ("SPH2D_LOG_TABLE_D", 2.0 ** -53)])
def test_table_entries(name, eps):
    rows = _entries(name)
    assert len(rows) == 128
    for i, (inv, hi, lo) in enumerate(rows):
        c = (64 + i) / 128.0
        assert abs(inv * c - 1.0) <= eps                  # 1/c_i rounded to the working precision
        assert abs((hi + lo) + math.log(inv)) <= 4 * eps * eps + 1e-300 + abs(math.log(inv)) * 1e-15
        assert abs(lo) <= abs(hi) * eps or hi == 0.0       # hi + lo is a normalised pair
    assert rows[64] == (1.0, 0.0, 0.0)                     # c = 1: no reduction near x = 1


PROG = r'''
#include <cmath>
#include <cstdio>
#include <random>
#include "pair_math.cuh"
using namespace sph2d;
int main() {
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> u(0, 1);
  double ef = 0, efn = 0, ed = 0;
  for (int k = 0; k < 300000; ++k) {
    double x;
    const int mode = k % 3;
    if (mode == 0) x = std::pow(10.0, -30 + 60 * u(g));
    else if (mode == 1) x = 1.0 + (u(g) - 0.5) * std::pow(10.0, -12 + 11 * u(g));
    else x = 0.5 + 1.5 * u(g);
    const float hi = float(x), lo = float(x - double(hi));
    const FF r = ff_log<float, float>(FF{hi, lo});
    const long double xf = (long double)hi + (long double)lo, ref = std::log(xf);
    const long double got = (long double)r.hi + (long double)r.lo;
    const double rel = double(std::fabs(got - ref) / std::fabs(ref));
    if (mode == 0) { if (double(std::fabs(got - ref)) > efn) efn = double(std::fabs(got - ref)); }
    else if (rel > ef) ef = rel;
    const FFT<double> rd = ff_log<double, double>(FFT<double>{x, 0.0});
    const long double refd = std::log((long double)x);
    const double reld = double(std::fabs(((long double)rd.hi + (long double)rd.lo) - refd) / std::fabs(refd));
    if (reld > ed) ed = reld;
  }
  std::printf("%.6e %.6e %.6e\n", ef, efn, ed);
  return 0;
}
'''


def test_compensated_log_accuracy(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "log.cpp"
    src.write_text(PROG)
    exe = tmp_path / "log"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    ef, efn, ed = map(float, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split())
    # float pairs: relative 2^-44 near and around 1 (where the result is small), absolute
    # 2e-12 over 60 decades (|ln x| up to 70 times the pair's relative precision: the e ln 2
    # term carries the ln 2 pair's rounding times e);
    # double pairs: long double's own precision (2^-64) bounds what this check can see
    assert ef < 6e-14, ef
    assert efn < 2e-12, efn
    assert ed < 3e-19, ed
