"""Pins for the surrogate reference (oracle/surrogate.py), each against something other than
itself: finite differences of the loss, geometric invariants of the canonical frame, the
exact inverse transform, a degenerate network with a known output, bfloat16 roundings
worked out by hand, and analytic integrals that the canonical frame must leave unchanged."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import surrogate as S


def glorot(rng):
    p = {}
    for name, shape in S.SHAPES:
        if name.startswith("W"):
            lim = math.sqrt(6.0 / (shape[0] + shape[1]))
            p[name] = rng.uniform(-lim, lim, size=shape)
        else:
            p[name] = rng.normal(0.0, 0.1, size=shape)
    return S.pack(p)


def random_local(rng, n, lo=0.12, hi=0.38):
    """triangles with a decent minimum angle placed inside the unit support."""
    out = []
    while len(out) < n:
        size = rng.uniform(lo, hi)
        ang = rng.uniform(0, 2 * np.pi)
        a = np.array([np.cos(ang), np.sin(ang)]) * size
        b = np.array([np.cos(ang + rng.uniform(1.0, 1.4)), np.sin(ang + rng.uniform(1.0, 1.4))]) * \
            size * rng.uniform(0.8, 1.0)
        c0 = rng.uniform(-0.7, 0.7, size=2)
        tri = np.array([c0, c0 + a, c0 + b])
        out.append(tri.ravel())
    return np.array(out)


def test_parameter_count():
    assert S.N_PARAMS == 8963


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(11)
    prm = glorot(rng)
    X = rng.uniform(-1, 1, size=(12, 6))
    T = rng.normal(size=(12, 3))
    w = np.array([1.0, 0.3, 0.7])
    L, g = S.loss_and_grad(prm, X, T, w)
    assert L == pytest.approx(S.loss(prm, X, T, w), rel=1e-14)
    # a sample of parameters from every tensor
    offs, o = [], 0
    for _, shape in S.SHAPES:
        n = int(np.prod(shape))
        offs += list(o + rng.choice(n, size=min(n, 6), replace=False))
        o += n
    h = 1e-6
    for i in offs:
        e = np.zeros_like(prm)
        e[i] = h
        fd = (S.loss(prm + e, X, T, w) - S.loss(prm - e, X, T, w)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_gelu_derivative_matches_differences():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (S.gelu(z + h) - S.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - S.gelu_grad(z))) < 1e-8
    # GELU(0) = 0, GELU(z) -> z for large z and -> 0 for very negative z
    assert S.gelu(np.array([0.0]))[0] == 0.0
    assert abs(S.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(S.gelu(np.array([-10.0]))[0]) < 1e-12


def test_f16_gelu_follows_gelu():
    """the stepwise FP16 GELU stays within a few FP16 steps of the exact one (relative, plus
    an absolute |z| 2^-12 where tanh rounds to -1 and the tail becomes 0), and has the exact
    limits (0 for very negative z, z for large z, including z^2 overflow)."""
    z = np.linspace(-12, 12, 4001)
    g, e = S.gelu_f16(z), S.gelu(S.f16(z))
    assert np.all(np.abs(g - e) <= 4e-3 * np.abs(e) + np.abs(z) * 2.0 ** -11)
    big = np.array([-300.0, -20.0, 20.0, 300.0, 1000.0])
    assert S.gelu_f16(big).tolist() == [0.0, 0.0, 20.0, 300.0, 1000.0]


def test_zero_weights_give_output_bias():
    p = S.unpack(np.zeros(S.N_PARAMS))
    p["b4"] = np.array([0.5, -1.25, 2.0])
    p["b1"] = np.full(64, 3.0)
    Y, _ = S.forward(S.pack(p), np.random.default_rng(0).normal(size=(5, 6)))
    assert np.array_equal(Y, np.tile(p["b4"], (5, 1)))


def test_f16_rounding_by_hand():
    # 11 significant bits: 2049 lies halfway between 2048 and 2050 -> even 2048
    assert S.f16(2049.0) == 2048.0 and S.f16(2051.0) == 2052.0
    assert S.f16(1.0 + 2.0 ** -11) == 1.0 and S.f16(1.0 + 2.0 ** -11 + 2.0 ** -20) == 1.0 + 2.0 ** -10
    assert S.f16(65504.0) == 65504.0 and S.f16(-0.5) == -0.5


def test_bf16_rounding_by_hand():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert S.bf16(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6 ... rounds to the even 1 + 2^-6
    assert S.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    # just above the halfway point rounds up
    assert S.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert S.bf16(-3.0) == -3.0
    assert S.bf16(0.0) == 0.0
    # 8 significant bits: 257 is not representable, 256 and 258 are
    assert S.bf16(257.0) == 256.0 and S.bf16(258.0) == 258.0


def _rot(theta):
    return np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])


def test_canonical_frame_invariants():
    rng = np.random.default_rng(5)
    loc = random_local(rng, 200)
    cn = S.canonicalize(loc)
    x = cn["x"].reshape(-1, 3, 2)
    c = x.mean(axis=1)
    # centroid on the +x axis, counter-clockwise, first vertex closest to the particle
    assert np.max(np.abs(c[:, 1])) < 1e-13
    assert np.all(c[:, 0] > 0)
    cr = (x[:, 1, 0] - x[:, 0, 0]) * (x[:, 2, 1] - x[:, 0, 1]) - (x[:, 1, 1] - x[:, 0, 1]) * (x[:, 2, 0] - x[:, 0, 0])
    assert np.all(cr > 0)
    d = np.hypot(x[..., 0], x[..., 1])
    assert np.all(d[:, 0] <= d[:, 1]) and np.all(d[:, 0] <= d[:, 2])
    # invariant under rotation about the particle, reflection and relabelling of the input
    for k in range(4):
        R = _rot(rng.uniform(0, 2 * np.pi))
        v = loc.reshape(-1, 3, 2) @ R.T
        if k % 2:
            v[..., 1] *= -1.0
        v = v[:, [2, 0, 1] if k < 2 else [1, 0, 2]]
        cn2 = S.canonicalize(v.reshape(-1, 6))
        assert np.max(np.abs(cn2["x"] - cn["x"])) < 1e-12
        assert np.array_equal(cn2["accept"], cn["accept"])


def test_inverse_transform_restores_triangle():
    rng = np.random.default_rng(6)
    loc = random_local(rng, 100)
    cn = S.canonicalize(loc)
    x = cn["x"].reshape(-1, 3, 2)
    # undo the reflection, then the rotation, vertex by vertex
    y = x.copy()
    y[..., 1] *= cn["refl"][:, None]
    back = np.empty_like(y)
    back[..., 0] = cn["cs"][:, None] * y[..., 0] - cn["sn"][:, None] * y[..., 1]
    back[..., 1] = cn["sn"][:, None] * y[..., 0] + cn["cs"][:, None] * y[..., 1]
    orig = loc.reshape(-1, 3, 2)
    for i in range(len(loc)):
        a = sorted(map(tuple, np.round(back[i], 12)))
        b = sorted(map(tuple, np.round(orig[i], 12)))
        assert np.allclose(a, b, atol=1e-12)
    # the gradient map is the transpose of the vertex map: a round trip is the identity
    g = rng.normal(size=(len(loc), 2))
    t = S.canonical_targets(cn, np.ones(len(loc)), g)
    back_g = S.uncanonicalize_grad(cn, t[:, 1:3] * cn["area"][:, None])
    assert np.max(np.abs(back_g - g)) < 1e-12


def test_canonical_frame_preserves_analytic_integrals():
    """gamma is invariant and the gradient equivariant under the canonical map (rotation
    and reflection about the particle): the oracle's integrals of the canonical triangle,
    mapped back, equal those of the input triangle."""
    rng = np.random.default_rng(7)
    loc = random_local(rng, 40)
    cn = S.canonicalize(loc)
    pa = np.zeros((len(loc), 8))
    pa[:, 2:] = loc
    pb = np.zeros((len(loc), 8))
    pb[:, 2:] = cn["x"]
    ra = oracle.pairs("wendland_c2", 1.0, pa)
    rb = oracle.pairs("wendland_c2", 1.0, pb)
    assert np.max(np.abs(ra[:, 0] - rb[:, 0])) < 1e-12
    g = S.uncanonicalize_grad(cn, rb[:, 1:3])
    assert np.max(np.abs(g - ra[:, 1:3])) < 1e-11


def test_guard_cases():
    def eq(side, centre):
        a = np.array([0.0, 0.0])
        b = np.array([side, 0.0])
        c = np.array([side / 2, side * math.sqrt(3) / 2])
        t = np.array([a, b, c])
        t = t - t.mean(axis=0) + np.asarray(centre)
        return t.ravel()

    tris = np.array([eq(0.3, (0.5, 0.2)),        # inside the domain
                     eq(0.05, (0.5, 0.2)),       # too small
                     eq(0.5, (0.5, 0.2)),        # too large
                     eq(0.3, (0.05, 0.05)),      # centroid too close to the particle
                     eq(0.3, (1.45, 0.0)),       # a vertex beyond 1.5 H
                     [0.5, 0.0, 0.8, 0.0, 0.65, 0.02]])   # sliver (smallest angle < 15 deg)
    acc = S.canonicalize(tris)["accept"]
    assert acc.tolist() == [True, False, False, False, False, False]
