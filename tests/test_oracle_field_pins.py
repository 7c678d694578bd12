"""Pins for the oracle's piecewise-linear boundary fields (Sec. 3, Eq. singleSpherical and
basicdiff), each against something other than the field quadrature itself: the paper's
full-cover test with a linear field (Sec. 6.2), the already-pinned gamma and grad gamma for a
constant field, central differences in the particle position, the moment route for the value,
and integration by parts with the transport-theorem vertex gradients for the gradient.  A
planted mutant (a lost power of r in the gradient density) must fail."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300.workloads import full_cover_square

KERNELS = ["wendland_c2", "wendland_c4", "wendland_c6", "cubic_spline"]


def lin(c0, cx, cy):
    return lambda x, y: c0 + cx * x + cy * y


def mesh_field(kernel, H, xp, tris, f, mutant=0):
    v, g = 0.0, np.zeros(2)
    for t in tris:
        vals = [f(t[0], t[1]), f(t[2], t[3]), f(t[4], t[5])]
        r = oracle.pair_field(kernel, H, xp, t, vals, mutant=mutant)
        v += r[0]
        g += r[1:]
    return v, g


@pytest.mark.parametrize("kernel", KERNELS)
def test_full_cover_linear_field(kernel):
    """Support inside [-1,1]^2 (the paper's 8-triangle mesh): <f> = f(x_i) and <grad f> is
    the field's gradient for any linear f; f = x at the centre gives 0 and [1, 0]."""
    tris = full_cover_square(2)
    v, g = mesh_field(kernel, 1.0, (0.0, 0.0), tris, lin(0.0, 1.0, 0.0))
    assert abs(v) < 1e-13 and np.allclose(g, [1.0, 0.0], atol=1e-12)
    v, g = mesh_field(kernel, 1.0, (0.0, 0.0), tris, lin(0.0, 0.0, 1.0))
    assert abs(v) < 1e-13 and np.allclose(g, [0.0, 1.0], atol=1e-12)
    f = lin(1.0, 2.0, -3.0)
    v, g = mesh_field(kernel, 0.5, (0.1, -0.05), tris, f)
    assert abs(v - f(0.1, -0.05)) < 1e-12 and np.allclose(g, [2.0, -3.0], atol=1e-11)


def random_pairs(rng, n, H=0.3):
    from paper_2507_21686_gb300 import workloads as W
    loc = W.surrogate_training_pairs(n, rng, lo=0.05, hi=1.5)
    xp = rng.uniform(-2, 2, size=(n, 2))
    pairs = np.zeros((n, 8))
    pairs[:, :2] = xp
    pairs[:, 2:] = loc[:, 2:] * H + np.tile(xp, 3)
    return pairs, H


@pytest.mark.parametrize("kernel", KERNELS)
def test_constant_field_is_gamma(kernel):
    rng = np.random.default_rng(31)
    pairs, H = random_pairs(rng, 60)
    vals = np.full((len(pairs), 3), 2.5)
    r = oracle.pairs_field(kernel, H, pairs, vals)
    ref = oracle.pairs(kernel, H, pairs)
    sg = 2.0 * np.max(np.abs(ref[:, 1:3])) + 1.0
    assert np.max(np.abs(r[:, 0] - 2.5 * ref[:, 0])) < 1e-12
    assert np.max(np.abs(r[:, 1:3] - 2.5 * ref[:, 1:3])) < 1e-11 * sg


@pytest.mark.parametrize("kernel", KERNELS)
def test_gradient_matches_central_differences(kernel):
    """the field stays fixed in world coordinates while the particle moves"""
    rng = np.random.default_rng(32)
    pairs, H = random_pairs(rng, 25)
    vals = rng.normal(size=(len(pairs), 3))
    h = 1e-6 * H
    r = oracle.pairs_field(kernel, H, pairs, vals)
    for c in range(2):
        pp, pm = pairs.copy(), pairs.copy()
        pp[:, c] += h
        pm[:, c] -= h
        fd = (oracle.pairs_field(kernel, H, pp, vals)[:, 0] - oracle.pairs_field(kernel, H, pm, vals)[:, 0]) / (2 * h)
        scale = np.maximum(np.abs(r[:, 1 + c]), 1.0 / H)
        assert np.max(np.abs(fd - r[:, 1 + c]) / scale) < 1e-6


def _linear_coeffs(tri, vals):
    """A(x) = c0 + c . x through the three vertices (world frame)"""
    Mx = np.array([[1.0, tri[0], tri[1]], [1.0, tri[2], tri[3]], [1.0, tri[4], tri[5]]])
    return np.linalg.solve(Mx, vals)


@pytest.mark.parametrize("kernel", KERNELS)
def test_value_by_moments_and_gradient_by_parts(kernel):
    """value = A(x_i) gamma + H grad A . (M10, M01); gradient = grad A gamma - sum_j A_j
    d gamma / d nu_j (integration by parts, transport-theorem edge integrals)"""
    rng = np.random.default_rng(33)
    pairs, H = random_pairs(rng, 40)
    vals = rng.normal(size=(len(pairs), 3))
    r = oracle.pairs_field(kernel, H, pairs, vals)
    ref = oracle.pairs(kernel, H, pairs)
    vg = oracle.pairs_vertex_grad(kernel, H, pairs)
    for i in range(len(pairs)):
        c0, cx, cy = _linear_coeffs(pairs[i, 2:], vals[i])
        a_i = c0 + cx * pairs[i, 0] + cy * pairs[i, 1]
        v = a_i * ref[i, 0] + H * (cx * ref[i, 6] + cy * ref[i, 7])
        g = np.array([cx, cy]) * ref[i, 0] - vals[i] @ vg[i].reshape(3, 2)
        s = 1.0 + np.max(np.abs(vals[i])) * (1.0 + np.abs(ref[i, 1:3]).max())
        assert abs(v - r[i, 0]) < 1e-11 * s, (i, v, r[i, 0])
        assert np.max(np.abs(g - r[i, 1:3])) < 1e-10 * s, (i, g, r[i, 1:3])


def test_mutant_is_caught():
    """a lost power of r in the gradient density fails the full-cover and difference pins"""
    oracle.build(mutant=5)
    tris = full_cover_square(2)
    _, g = mesh_field("wendland_c2", 1.0, (0.0, 0.0), tris, lin(0.0, 1.0, 0.0), mutant=5)
    assert not np.allclose(g, [1.0, 0.0], atol=1e-6)
