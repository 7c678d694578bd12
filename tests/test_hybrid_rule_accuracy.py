"""The hybrid mode's quadrature rule for the cubic spline's second piece, in exact (FP64)
arithmetic against the oracle on the CPU: for a near pair (triangle within H/2 of the particle,
not inside r < H/2, innermost vertex inside r < H/2, longest edge below 0.45 H, at least half its
longest edge from the particle), the first piece by the 6 x 6 conical rule and the second by a
10-ray rule of 6 nodes per ray in the doubled frame, where that piece's support is the unit
disk, give every output within 1e-6 of its scale; 6 rays do not.  This pins the rule's sizes
independently of the GPU (whose FP32 evaluation of the same rule is tested in
test_gpu_hybrid.py)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300 import workloads as W
from tests.helpers import scales

MA = [0, 1, 0, 2, 1, 0, 3, 2, 1, 0]
MB = [0, 0, 1, 0, 1, 2, 0, 1, 2, 3]


def _cross(a, b):
    return a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]


def _seg_dist(a, b):
    e = b - a
    t = np.clip(-(a * e).sum(-1) / (e * e).sum(-1), 0.0, 1.0)
    p = a + t[:, None] * e
    return np.hypot(p[:, 0], p[:, 1])


def near_class(count, seed):
    """local triangles (H = 1) of the class, innermost vertex first"""
    rng = np.random.default_rng(seed)
    loc = W.surrogate_training_pairs(40 * count, rng, lo=0.05, hi=0.6)[:, 2:].reshape(-1, 3, 2)
    v0, v1, v2 = loc[:, 0], loc[:, 1], loc[:, 2]
    dist = np.minimum.reduce([_seg_dist(v0, v1), _seg_dist(v1, v2), _seg_dist(v2, v0)])
    c = np.stack([_cross(v0, v1), _cross(v1, v2), _cross(v2, v0)], 1)
    inside = np.all(c > 0, 1) | np.all(c < 0, 1)
    r = np.hypot(loc[..., 0], loc[..., 1])
    lmax = np.max([np.hypot(*(loc[:, (i + 1) % 3] - loc[:, i]).T) for i in range(3)], axis=0)
    sel = (~inside & (dist >= 0.5 * lmax) & (dist < 0.5) & (r.max(1) >= 0.5) & (r.min(1) < 0.5)
           & (lmax < 0.45))
    loc, r = loc[sel][:count], r[sel][:count]
    assert len(loc) == count
    o = np.argmin(r, 1)
    return np.stack([loc[np.arange(len(loc)), (o + j) % 3] for j in range(3)], 1)


def conical(L, n_rays, k, dk):
    """integrals over the triangles L [n, 3, 2] (apex L[:, 0] inside the unit disk) of k(r),
    k'(r) p / r and k(r) p^m, with rays cut at r = 1: n_rays rays, 6 Gauss-Legendre nodes each"""
    x, w = np.polynomial.legendre.leggauss(n_rays)
    ut, wt = (x + 1) / 2, w / 2
    x, w = np.polynomial.legendre.leggauss(6)
    us, ws = (x + 1) / 2, w / 2
    v0, v1, v2 = L[:, 0], L[:, 1], L[:, 2]
    a2 = np.abs(_cross(v1 - v0, v2 - v0))
    out = np.zeros((len(L), 13))
    for tj, wj in zip(ut, wt):
        d = (v1 - v0) + tj * (v2 - v1)
        a, b, c = (d * d).sum(1), (v0 * d).sum(1), (v0 * v0).sum(1) - 1.0
        smax = np.minimum(1.0, (-b + np.sqrt(b * b - a * c)) / a)
        for si, wi in zip(us, ws):
            s = smax * si
            p = v0 + s[:, None] * d
            r = np.hypot(p[:, 0], p[:, 1])
            jac = wj * wi * smax * s * a2
            kv, dkv = k(r), dk(r)
            out[:, 0] += jac * kv
            out[:, 1] += jac * dkv * p[:, 0] / r
            out[:, 2] += jac * dkv * p[:, 1] / r
            for m, (ea, eb) in enumerate(zip(MA, MB)):
                out[:, 3 + m] += jac * kv * p[:, 0] ** ea * p[:, 1] ** eb
    return out


def k1(r):
    return np.where(r < 1, (1 - np.minimum(r, 1)) ** 3, 0.0)


def dk1(r):
    return np.where(r < 1, -3 * (1 - np.minimum(r, 1)) ** 2, 0.0)


def rule_error(L, n_rays):
    """max over the pairs of the largest output error relative to its scale"""
    C = oracle.kernel_C("cubic_spline")
    p1 = conical(L, 6, k1, dk1)                 # first piece 2 k1(r)
    p2 = conical(2.0 * L, n_rays, k1, dk1)      # second piece k1(2 r), doubled frame
    deg = np.array(MA) + np.array(MB)
    got = np.zeros_like(p1)
    got[:, 0] = C * (2 * p1[:, 0] - 0.25 * p2[:, 0])
    got[:, 1:3] = -C * (2 * p1[:, 1:3] - 0.5 * p2[:, 1:3])
    for m in range(10):
        got[:, 3 + m] = C * (2 * p1[:, 3 + m] - 2.0 ** (-(deg[m] + 2)) * p2[:, 3 + m])
    pairs = np.zeros((len(L), 8))
    pairs[:, 2:] = L.reshape(-1, 6)
    ref = oracle.pairs("cubic_spline", 1.0, pairs)
    ref = np.concatenate([ref[:, :3], ref[:, 5:15]], 1)
    return (np.abs(got - ref) / np.maximum(np.abs(ref), scales("cubic_spline", 1.0, 10))).max()


@pytest.fixture(scope="module")
def tris():
    return near_class(1500, 7)


def test_ten_rays_within_1e6(tris):
    assert rule_error(tris, 10) <= 1e-6


def test_six_rays_are_not_enough(tris):
    """the kink of (1 - r')^3_+ at r' = 1 runs across the rays, so their number sets the error"""
    assert rule_error(tris, 6) > 2e-6
