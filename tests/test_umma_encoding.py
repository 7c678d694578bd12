"""CPU checks of the tcgen05 descriptor encoders in csrc/umma.cuh against the PTX ISA field
layouts (shared-memory matrix descriptor and the kind::f16 instruction descriptor), and of the
K-major no-swizzle core-matrix offsets.  The encoders are compiled for the host with g++ and
their outputs decoded here field by field."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2507_21686_gb300", "csrc", "umma.cuh")

PROG = r'''
#include <cstdio>
#include "umma.cuh"
using namespace sph2d::umma;
int main() {
  const unsigned addrs[] = {0u, 1024u, 0x12340u, 0x3fff0u};
  const unsigned lbos[] = {128u, 1024u, 256u};
  const unsigned sbos[] = {1024u, 128u, 2048u};
  for (unsigned a : addrs) for (int i = 0; i < 3; ++i)
    std::printf("S %u %u %u %llu\n", a, lbos[i], sbos[i], (unsigned long long)smem_desc(a, lbos[i], sbos[i]));
  const unsigned Ms[] = {64u, 128u}, Ns[] = {16u, 64u, 256u};
  for (unsigned m : Ms) for (unsigned n : Ns) for (int b = 0; b < 2; ++b)
    std::printf("I %u %u %d %u\n", m, n, b, idesc_f16(m, n, b != 0));
  for (unsigned r = 0; r < 16; ++r) for (unsigned c = 0; c < 64; c += 3)
    std::printf("O %u %u %u\n", r, c, kmajor_offset(r, c, 64));
  return 0;
}
'''


def bits(v, lo, hi):
    """bits lo..hi inclusive"""
    return (v >> lo) & ((1 << (hi - lo + 1)) - 1)


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("umma")
    src = d / "enc.cpp"
    src.write_text(PROG)
    exe = d / "enc"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")


def test_smem_descriptor_fields(lines):
    rows = [l.split() for l in lines if l.startswith("S ")]
    assert len(rows) == 12
    for _, a, lbo, sbo, d in rows:
        a, lbo, sbo, d = int(a), int(lbo), int(sbo), int(d)
        assert bits(d, 0, 13) == (a >> 4) & 0x3FFF          # start address, 16-byte units
        assert bits(d, 14, 15) == 0
        assert bits(d, 16, 29) == lbo >> 4                  # leading-dimension byte offset
        assert bits(d, 30, 31) == 0
        assert bits(d, 32, 45) == sbo >> 4                  # stride-dimension byte offset
        assert bits(d, 46, 47) == 1                         # descriptor version of sm_100-class GPUs
        assert bits(d, 48, 48) == 0
        assert bits(d, 49, 51) == 0                         # base offset
        assert bits(d, 52, 52) == 0                         # LBO mode
        assert bits(d, 53, 60) == 0
        assert bits(d, 61, 63) == 0                         # no swizzle


def test_instruction_descriptor_fields(lines):
    rows = [l.split() for l in lines if l.startswith("I ")]
    assert len(rows) == 12
    for _, m, n, bf, d in rows:
        m, n, bf, d = int(m), int(n), int(bf), int(d)
        assert bits(d, 0, 3) == 0                           # dense, no saturation
        assert bits(d, 4, 5) == 1                           # D format F32
        assert bits(d, 6, 6) == 0
        assert bits(d, 7, 9) == bf                          # A format: 0 F16, 1 BF16
        assert bits(d, 10, 12) == bf                        # B format
        assert bits(d, 13, 14) == 0                         # no negation
        assert bits(d, 15, 16) == 0                         # A and B K-major
        assert bits(d, 17, 22) == n >> 3                    # N / 8
        assert bits(d, 23, 23) == 0
        assert bits(d, 24, 28) == m >> 4                    # M / 16
        assert bits(d, 29, 31) == 0
    assert d < 2 ** 32


def test_core_matrix_offsets(lines):
    """K-major, no swizzle: 8 x 8 core matrices of 128 contiguous bytes (rows of 16 bytes),
    column groups 128 bytes apart, row groups 128 K / 8 bytes apart; distinct elements never
    share a byte and the 16 x 64 block fills exactly its 2 KB"""
    rows = [tuple(map(int, l.split()[1:])) for l in lines if l.startswith("O ")]
    seen = set()
    for r, c, off in rows:
        assert off == (r // 8) * 1024 + (c // 8) * 128 + (r % 8) * 16 + (c % 8) * 2
        assert off % 2 == 0 and off < 16 * 64 * 2
        assert off not in seen
        seen.add(off)
