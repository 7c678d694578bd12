"""Error metrics of the accuracy targets, shared by the tests and bench.py.

Two relative errors, both against a reference b (the FP64 oracle or the FP64 GPU path):

    per-particle sums   err(a, b) = |a - b| / max(|b|, S_r)
    per pair            err(a, b) = |a - b| / max(|b|, 1e-6 S_r)

S_r is the natural full-support scale of output r for kernel k and support H:
    gamma      S = 1                                  (int W over the whole support)
    grad       S = 2 C int_0^1 k(q) dq / H            (|grad gamma| at a straight wall)
    M_ab       S = C int_disc |xi^a eta^b| k dA       (absolute moment over the support)

A per-particle sum is O(S_r) wherever the boundary matters, so values at least as large as
their scale are compared relatively and smaller ones in units of the scale.  A single pair's
value can be many decades smaller (a triangle of 1e-3 H has gamma ~ 1e-6), so per-pair values
are compared relatively down to 1e-6 of the scale.  Targets: FP64 path 1e-10, FP32 path 1e-5,
learned surrogate 1e-3.  The scales are exact rationals of the kernel polynomials (plus pi).
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np

TOL_FP64 = 1e-10
TOL_FP32 = 1e-5
TOL_SURROGATE = 1e-3
PAIR_FLOOR = 1e-6


def _pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += Fr(x) * Fr(y)
    return out


def _ppow(a, n):
    out = [Fr(1)]
    for _ in range(n):
        out = _pmul(out, a)
    return out


_OMQ = [Fr(1), Fr(-1)]
_PIECES = {
    "wendland_c2": [(_pmul(_ppow(_OMQ, 4), [1, 4]), Fr(0), Fr(1))],
    "wendland_c4": [(_pmul(_ppow(_OMQ, 6), [1, 6, Fr(35, 3)]), Fr(0), Fr(1))],
    "wendland_c6": [(_pmul(_ppow(_OMQ, 8), [1, 8, 25, 32]), Fr(0), Fr(1))],
    "cubic_spline": [([Fr(1), Fr(0), Fr(-6), Fr(6)], Fr(0), Fr(1, 2)),
                     (_pmul([2], _ppow(_OMQ, 3)), Fr(1, 2), Fr(1))],
}
KERNEL_NAMES = ["wendland_c2", "wendland_c4", "wendland_c6", "cubic_spline"]


def radial_moment(kernel, p):
    """int_0^1 q^p k(q) dq, exactly."""
    tot = Fr(0)
    for coef, lo, hi in _PIECES[kernel]:
        for k, b in enumerate(coef):
            n = k + p + 1
            tot += b * (hi ** n - lo ** n) / n
    return float(tot)


# int_0^{2 pi} |cos^a sin^b| dtheta
_ANG = {(0, 0): 2 * math.pi, (1, 0): 4.0, (0, 1): 4.0, (2, 0): math.pi, (1, 1): 2.0,
        (0, 2): math.pi, (3, 0): 8.0 / 3.0, (2, 1): 4.0 / 3.0, (1, 2): 4.0 / 3.0, (0, 3): 8.0 / 3.0}
MOMENT_ORDER = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3)]


def scales(kernel, H: float, nm: int = 10) -> np.ndarray:
    """Scales for (gamma, gx, gy, M00..M_{nm-1})."""
    if isinstance(kernel, int):
        kernel = KERNEL_NAMES[kernel]
    C = 1.0 / (2.0 * math.pi * radial_moment(kernel, 1))
    sg = 2.0 * C * radial_moment(kernel, 0) / H
    sm = [C * _ANG[ab] * radial_moment(kernel, 1 + ab[0] + ab[1]) for ab in MOMENT_ORDER[:nm]]
    return np.array([1.0, sg, sg] + sm)


def rel_err(a, b, scale) -> np.ndarray:
    """|a - b| / max(|b|, scale), elementwise (scale broadcast over the last axis)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), scale)


def pair_rel_err(a, b, scale) -> np.ndarray:
    """Per-pair relative error: |a - b| / max(|b|, 1e-6 scale)."""
    return rel_err(a, b, PAIR_FLOOR * np.asarray(scale, dtype=np.float64))
