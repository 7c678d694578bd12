#!/usr/bin/env python3
"""Writes log_table.h: the argument-reduction table of the compensated natural logarithm in
pair_math.cuh (ff_log).  Entry i (0..127) is for mantissas m in [1/sqrt2, sqrt2) nearest to
c_i = (64 + i)/128 (entries 27..117 are reached; c_64 = 1):
    inv  = 1/c_i rounded to the working precision (float or double), an exact machine number
    L    = -ln(inv), exactly for that machine number, to 60 decimal digits, split into hi + lo
           of the working precision (hi = L rounded, lo = (L - hi) rounded)
so that ln(m) = L + ln(m * inv) with m * inv within 2^-7.5 of 1, and m * inv - 1 = m - 1 exactly at c = 1.  Run from this directory:
    python gen_log_table.py > log_table.h
"""
from decimal import Decimal, getcontext

import numpy as np

getcontext().prec = 60


def split(v: Decimal, ftype):
    hi = ftype(float(v))
    lo = ftype(float(v - Decimal(float(hi))))
    return hi, lo


def main():
    rows_f, rows_d = [], []
    for i in range(128):
        c = (64 + i) / 128.0
        inv_f = np.float32(1.0) / np.float32(c)
        inv_d = 1.0 / c
        lf = -Decimal(float(inv_f)).ln()
        ld = -Decimal(inv_d).ln()
        hf, lof = split(lf, np.float32)
        hd, lod = split(ld, np.float64)
        rows_f.append(f"{{{float(inv_f).hex()}f, {float(hf).hex()}f, {float(lof).hex()}f}}")
        rows_d.append(f"{{{float(inv_d).hex()}, {float(hd).hex()}, {float(lod).hex()}}}")
    print("// Generated by gen_log_table.py: {1/c_i, -ln(1/c_i) hi, lo}, c_i = (64 + i)/128, i = 0..127,")
    print("// in float (LOG_TABLE_F) and double (LOG_TABLE_D); -ln exact to 60 digits for the stored 1/c_i.")
    print("#pragma once")
    print("#define SPH2D_LOG_TABLE_F \\")
    print(", \\\n".join("  " + r for r in rows_f))
    print("#define SPH2D_LOG_TABLE_D \\")
    print(", \\\n".join("  " + r for r in rows_d))


if __name__ == "__main__":
    main()
