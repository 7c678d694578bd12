"""CPU pins of the grid-extraction sums of the FP32 closed form (csrc/pair_math.cuh): the
per-fan power-of-two scale, the exactness of the extracted running sum and its absolute error
bound (checked against exact rational arithmetic), and the per-slot grid constants against the
coefficient rows they must bound.  The header is compiled for the host with g++."""
from __future__ import annotations

import math
import os
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2507_21686_gb300", "csrc")

PROG = r'''
#include <cmath>
#include <cstdio>
#include <random>
#include "pair_math.cuh"
using namespace sph2d;

template <class P>
static void grids(const char* name) {
  for (int s = 0; s < NSL; ++s) {
    std::printf("G %s %d %a %d %a", name, s, double(slot_grid<P>(s)), int(slot_uses_drho(s)), poly_scale<P>());
    for (int q = -1; q <= P::K + 4; ++q) {
      const NumDen c = edge_coef<P>(q, s);
      if (c.num != 0.0) std::printf(" %d:%a:%a", q, c.num, c.den);
    }
    std::printf("\n");
  }
  std::printf("M %s %d\n", name, int(uses_row_m1<P>()));
  std::printf("D %s %lld\n", name, poly_den<P>());
  for (int q = -1; q <= P::K + 4; ++q)
    for (int s = 0; s < NSL; ++s) {
      const NumDen c = edge_coef_y<P>(q, s);
      if (c.num != 0.0)
        std::printf("E %s %d %d %a %a\n", name, q, s, double(float(edge_coef_s<P>(q, s))), c.num / c.den);
    }
}

int main() {
  grids<PolyWC2>("wc2");
  grids<PolyWC4>("wc4");
  grids<PolyWC6>("wc6");
  grids<PolyCube>("cube");
  std::mt19937_64 g(11);
  std::uniform_real_distribution<double> u(-1, 1);
  // sums of n products with |x k| <= grid / (2n), alternating signs so that the exact sum cancels
  for (int trial = 0; trial < 400; ++trial) {
    const int n = 2 + trial % 15;
    const float grid = std::ldexp(1.0f, -20 + int(trial % 41));
    CSum<float> acc = xsum_init<float>(grid);
    std::printf("S %d %a", n, double(grid));
    for (int i = 0; i < n; ++i) {
      const double kv = (1.0 + 3.0 * std::fabs(u(g))) * ((i & 1) ? -1 : 1);
      const FF k = ff_const(trial % 3 == 0 ? double(float(kv)) : kv);
      const double xv = u(g) * double(grid) / (n * 8.0);
      const float xh = float(xv), xl = float(xv - double(xh));
      acc = xsum_madd(acc, FF{xh, xl}, k.hi, k.lo);
      std::printf(" %a,%a,%a,%a", double(xh), double(xl), double(k.hi), double(k.lo));
    }
    const FF r = xsum_result(acc, grid);
    std::printf(" | %a %a %a %a\n", double(acc.s - 1.5f * grid), double(acc.c), double(r.hi), double(r.lo));
  }
  // the scale: 2^-e with |x| in [2^(e-1), 2^e)
  for (int i = 0; i < 2000; ++i) {
    float x;
    if (i < 300) x = std::ldexp(1.0f, -70 + i % 100);                   // powers of two
    else if (i < 400) x = std::nextafter(std::ldexp(1.0f, -30 + i % 60), 0.0f);
    else if (i < 420) x = std::ldexp(1.0f, -140 + i % 20);              // subnormal
    else x = float(std::exp(40.0 * u(g))) * (i & 1 ? -1.0f : 1.0f);
    const Pow2<float> p = pow2_scale(x);
    std::printf("P %a %a %a\n", double(x), double(p.s), double(p.is));
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("gridsum")
    src = d / "gs.cpp"
    src.write_text(PROG)
    exe = d / "gs"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()


def is_pow2(v):
    m, _ = math.frexp(v)
    return v > 0 and m == 0.5


def test_slot_grids_bound_their_terms(lines):
    """every slot's grid g is a power of two with g >= 2 n m and g < 4 n m (1 + 2^-7), where n
    counts the non-zero rows and m is the largest |coefficient| times its input bound (1 for
    Delta J_q, q for Delta rho^q) times the polynomial's FP32 scale D_P"""
    rows = [l.split() for l in lines if l.startswith("G ")]
    assert len(rows) == 4 * 12
    for r in rows:
        g, drho, scale = float.fromhex(r[3]), r[4] == "1", float.fromhex(r[5])
        terms = [t.split(":") for t in r[6:]]
        if not terms:
            continue
        n = len(terms)
        m = 0.0
        for q, num, den in terms:
            q = int(q)
            w = abs(float.fromhex(num)) / float.fromhex(den) * (q if drho and q > 1 else 1)
            m = max(m, w)
        need = 2 * n * m * scale                        # the FP32 rows run times D_P
        assert is_pow2(g), r
        assert g >= need, r
        assert g < 2 * need * (1 + 2 ** -7), r
        if drho:
            assert all(int(q) >= 1 for q, _, _ in terms), r     # Delta rho^q rows start at q = 1


def test_row_minus_one_only_with_a_linear_term(lines):
    """the q = -1 row (Delta J_-1, the unbounded log term) is used only by the cubic spline,
    whose (1 - q)^3 has a linear term; Wendland kernels have b_1 = 0"""
    flags = dict((l.split()[1], l.split()[2]) for l in lines if l.startswith("M "))
    assert flags == {"wc2": "0", "wc4": "0", "wc6": "0", "cube": "1"}


def test_extracted_sum_error_bound(lines):
    """the running-sigma sum, started at 3g/2: s - 3g/2 (exact) plus c against the exact rational
    sum of (x.hi + x.lo)(k.hi + k.lo), within 4 n^2 u^2 g absolute (u = 2^-24), far below the
    u g that a rounded running sum would show; s - 3g/2 is a multiple of 2 u g with
    |s - 3g/2| <= g/2, and the returned pair is s - 3g/2 + c to one rounding"""
    rows = [l for l in lines if l.startswith("S ")]
    assert len(rows) == 400
    u = Fraction(1, 2 ** 24)
    worst = 0.0
    for l in rows:
        head, tail = l[2:].split(" | ")
        parts = head.split()
        n, g = int(parts[0]), Fraction(float.fromhex(parts[1]))
        exact = Fraction(0)
        for t in parts[2:]:
            xh, xl, kh, kl = (Fraction(float.fromhex(v)) for v in t.split(","))
            exact += (xh + xl) * (kh + kl)
        s, c, rh, rl = (Fraction(float.fromhex(v)) for v in tail.split())
        assert abs(s) <= g / 2
        assert (s / (2 * u * g)).denominator == 1
        assert rh + rl == s + c or abs(rh + rl - (s + c)) <= u * u * abs(s + c)
        err = abs(s + c - exact)
        bound = 4 * n * n * u * u * g
        assert err <= bound, (l, float(err), float(bound))
        worst = max(worst, float(err / (u * u * g)))
    assert worst > 0.0                                          # the check can see an error


def test_pow2_scale(lines):
    rows = [l.split() for l in lines if l.startswith("P ")]
    assert len(rows) == 2000
    for _, x, s, i in rows:
        x, s, i = float.fromhex(x), float.fromhex(s), float.fromhex(i)
        assert is_pow2(s) and is_pow2(i) and s * i == 1.0
        assert s <= 2.0 ** 64
        if s < 2.0 ** 64:
            assert 0.5 <= abs(x) * s < 1.0, (x, s)
        else:
            assert abs(x) * s < 1.0, (x, s)


# kernel polynomials k(q) = sum_k b_k q^k from their factored definitions (Wendland C2, C4, C6
# and the cubic spline's (1 - q)^3 piece), in exact rationals
def _poly_mul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _poly_pow(a, n):
    out = [Fraction(1)]
    for _ in range(n):
        out = _poly_mul(out, a)
    return out


_ONE_MINUS_Q = [Fraction(1), Fraction(-1)]
POLYS = {
    "wc2": _poly_mul(_poly_pow(_ONE_MINUS_Q, 4), [Fraction(1), Fraction(4)]),
    "wc4": _poly_mul(_poly_pow(_ONE_MINUS_Q, 6), [Fraction(1), Fraction(6), Fraction(35, 3)]),
    "wc6": _poly_mul(_poly_pow(_ONE_MINUS_Q, 8), [Fraction(1), Fraction(8), Fraction(25), Fraction(32)]),
    "cube": _poly_pow(_ONE_MINUS_Q, 3),
}


def _odd(v):
    v = abs(v)
    while v and v % 2 == 0:
        v //= 2
    return v


def test_exact_fp32_rows(lines):
    """the FP32 path's scaled rows: D_P is the odd part of the least common multiple of the row
    denominators, every scaled entry is exactly D_P times the row's rational value (so exact in
    FP32, no low word), and D_P is 0 (float-pair rows kept) exactly where some scaled numerator
    would need more than 24 bits (Wendland C6)"""
    den = {l.split()[1]: int(l.split()[2]) for l in lines if l.startswith("D ")}
    assert set(den) == set(POLYS)
    for name, b in POLYS.items():
        rows = [l.split() for l in lines if l.startswith("E " + name + " ")]
        assert rows
        vals = []
        for r in rows:
            v = Fraction(float.fromhex(r[5])).limit_denominator(10 ** 9)
            assert abs(float(v) - float.fromhex(r[5])) <= 1e-15 * abs(float(v))
            vals.append((int(r[2]), int(r[3]), v, float.fromhex(r[4])))
        lcm = 1
        for _, _, v, _ in vals:
            lcm = lcm * _odd(v.denominator) // math.gcd(lcm, _odd(v.denominator))
        fits = all(_odd((v * lcm).numerator) < 2 ** 24 for _, _, v, _ in vals)
        assert den[name] == (lcm if fits else 0), name
        # the leading row of gamma (q = 0, slot 0): b_0 / 2 of the factored polynomial
        g0 = [v for q, s, v, _ in vals if q == 0 and s == 0]
        assert g0 == [b[0] / 2], name
        for q, s, v, scaled in vals:
            if den[name] == 0:
                assert scaled == 0.0
            else:
                assert Fraction(scaled) == v * den[name], (name, q, s)
