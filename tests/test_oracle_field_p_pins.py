"""Pins for the oracle's Lagrange (P2, P3) boundary fields, each against something other than
the nodal field quadrature itself: the linear-field oracle (a different route: the field
expanded as a0 + a . p), exact reproduction of lower-order fields, the full-cover closed forms
for quadratic and cubic fields (Sec. 6.2's full-cover mesh, extended: with the support inside
the mesh, <f> = f(x_i) + H^2 m2 (second derivatives) and <grad f> = <grad of f>), central
differences in the particle position, and the moment route for the value.  A planted mutant
(two edge nodes of P3 swapped) must fail."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300.workloads import full_cover_square

KERNELS = ["wendland_c2", "wendland_c4", "wendland_c6", "cubic_spline"]


def kernel_second_moment(kernel):
    """m2 = int_{R^2} xi^2 W(|xi|) d xi (H = 1) = C pi int_0^1 r^3 k(r) dr, from the kernels'
    factored definitions (Sec. 2) and their 2-D normalisation int W = 1, both by Gauss-Legendre
    of the exact polynomial pieces (independent of the oracle's code)."""
    x, w = np.polynomial.legendre.leggauss(30)

    def k(r):
        if kernel == "wendland_c2":
            return (1 - r) ** 4 * (1 + 4 * r)
        if kernel == "wendland_c4":
            return (1 - r) ** 6 * (1 + 6 * r + 35 / 3 * r * r)
        if kernel == "wendland_c6":
            return (1 - r) ** 8 * (1 + 8 * r + 25 * r * r + 32 * r ** 3)
        return np.where(r < 0.5, 1 - 6 * r * r + 6 * r ** 3, 2 * (1 - r) ** 3)

    def integ(f):
        pieces = [(0.0, 0.5), (0.5, 1.0)]
        return sum(0.5 * (b - a) * np.sum(w * f(0.5 * (b - a) * x + 0.5 * (a + b))) for a, b in pieces)

    norm = 2 * np.pi * integ(lambda r: k(r) * r)        # int k dA; C = 1 / norm
    return np.pi * integ(lambda r: k(r) * r ** 3) / norm


def mesh_field_p(kernel, H, xp, tris, order, f, mutant=0):
    v, g = 0.0, np.zeros(2)
    nodes = oracle.field_nodes(tris, order)
    for t, nd in zip(tris, nodes):
        r = oracle.pair_field_p(kernel, H, xp, t, order, f(nd[:, 0], nd[:, 1]), mutant=mutant)
        v += r[0]
        g += r[1:]
    return v, g


FIELDS = {
    # f, its gradient, <f> and <grad f> for a full cover at particle (x, y), H, m2
    "x2": (lambda x, y: x * x, lambda x, y, s: (x * x + s, (2 * x, 0.0))),
    "xy": (lambda x, y: x * y, lambda x, y, s: (x * y, (y, x))),
    "y2+x": (lambda x, y: y * y + x, lambda x, y, s: (y * y + s + x, (1.0, 2 * y))),
    "x3": (lambda x, y: x ** 3, lambda x, y, s: (x ** 3 + 3 * x * s, (3 * (x * x + s), 0.0))),
    "x2y": (lambda x, y: x * x * y, lambda x, y, s: (x * x * y + y * s, (2 * x * y, x * x + s))),
    "y3-xy2": (lambda x, y: y ** 3 - x * y * y,
               lambda x, y, s: (y ** 3 + 3 * y * s - x * (y * y + s), (-(y * y + s), 3 * (y * y + s) - 2 * x * y))),
}


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("name", list(FIELDS))
def test_full_cover_polynomial_fields(kernel, name):
    """quadratic fields on P2 and P3 elements, cubic fields on P3 elements: exact closed forms
    (s = H^2 m2 is the kernel's second moment)"""
    f, ref = FIELDS[name]
    cubic = name in ("x3", "x2y", "y3-xy2")
    tris = full_cover_square(2)
    H, xp = 0.5, (0.1, -0.05)
    s = H * H * kernel_second_moment(kernel)
    rv, rg = ref(xp[0], xp[1], s)
    for order in ((3,) if cubic else (2, 3)):
        v, g = mesh_field_p(kernel, H, xp, tris, order, f)
        assert abs(v - rv) < 1e-12, (order, v, rv)
        assert np.allclose(g, rg, atol=1e-11), (order, g, rg)


def random_pairs(rng, n, H=0.3):
    from paper_2507_21686_gb300 import workloads as W
    loc = W.surrogate_training_pairs(n, rng, lo=0.05, hi=1.5)
    xp = rng.uniform(-2, 2, size=(n, 2))
    pairs = np.zeros((n, 8))
    pairs[:, :2] = xp
    pairs[:, 2:] = loc[:, 2:] * H + np.tile(xp, 3)
    return pairs, H


def node_values(pairs, order, f):
    nd = oracle.field_nodes(pairs[:, 2:], order)
    return f(nd[..., 0], nd[..., 1])


@pytest.mark.parametrize("kernel", KERNELS)
def test_lower_order_fields_reproduced(kernel):
    """a linear field on P2/P3 nodes equals the linear-field oracle (field expanded as
    a0 + a . p there); a quadratic field on P3 nodes equals it on P2 nodes"""
    rng = np.random.default_rng(41)
    pairs, H = random_pairs(rng, 40)
    c = rng.normal(size=6)
    lin = lambda x, y: c[0] + c[1] * x + c[2] * y
    quad = lambda x, y: lin(x, y) + c[3] * x * x + c[4] * x * y + c[5] * y * y
    ref = oracle.pairs_field(kernel, H, pairs, node_values(pairs, 1, lin))
    sc = 1.0 + np.abs(ref).max(axis=1, keepdims=True)
    for order in (1, 2, 3):
        got = oracle.pairs_field_p(kernel, H, pairs, order, node_values(pairs, order, lin))
        assert np.max(np.abs(got - ref) / sc) < 1e-12, order
    r2 = oracle.pairs_field_p(kernel, H, pairs, 2, node_values(pairs, 2, quad))
    r3 = oracle.pairs_field_p(kernel, H, pairs, 3, node_values(pairs, 3, quad))
    assert np.max(np.abs(r2 - r3) / (1.0 + np.abs(r2).max(axis=1, keepdims=True))) < 1e-12


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("order", [2, 3])
def test_gradient_matches_central_differences(kernel, order):
    """the field stays fixed in world coordinates while the particle moves"""
    rng = np.random.default_rng(42 + order)
    pairs, H = random_pairs(rng, 20)
    vals = rng.normal(size=(len(pairs), oracle.nodes_per_triangle(order)))
    h = 1e-6 * H
    r = oracle.pairs_field_p(kernel, H, pairs, order, vals)
    for c in range(2):
        pp, pm = pairs.copy(), pairs.copy()
        pp[:, c] += h
        pm[:, c] -= h
        fd = (oracle.pairs_field_p(kernel, H, pp, order, vals)[:, 0]
              - oracle.pairs_field_p(kernel, H, pm, order, vals)[:, 0]) / (2 * h)
        scale = np.maximum(np.abs(r[:, 1 + c]), np.abs(vals).max(axis=1) / H)
        assert np.max(np.abs(fd - r[:, 1 + c]) / scale) < 1e-6


@pytest.mark.parametrize("kernel", KERNELS)
def test_value_by_moments(kernel):
    """<A> = sum_ab c_ab M_ab with c the monomial coefficients of the interpolant in the local
    frame (here by solving the 10 x 10 interpolation system at the P3 nodes) and M_ab the
    oracle's pinned moments"""
    rng = np.random.default_rng(44)
    pairs, H = random_pairs(rng, 30)
    vals = rng.normal(size=(len(pairs), 10))
    r = oracle.pairs_field_p(kernel, H, pairs, 3, vals)
    mom = oracle.pairs(kernel, H, pairs)[:, 5:15]
    nodes = oracle.field_nodes(pairs[:, 2:], 3)
    ea = [0, 1, 0, 2, 1, 0, 3, 2, 1, 0]
    eb = [0, 0, 1, 0, 1, 2, 0, 1, 2, 3]
    for i in range(len(pairs)):
        loc = (nodes[i] - pairs[i, :2]) / H
        V = np.stack([loc[:, 0] ** a * loc[:, 1] ** b for a, b in zip(ea, eb)], axis=1)
        c = np.linalg.solve(V, vals[i])
        v = c @ mom[i]
        s = 1.0 + np.abs(c).max() * np.abs(mom[i]).max()
        assert abs(v - r[i, 0]) < 1e-10 * s, (i, v, r[i, 0])


def test_mutant_is_caught():
    """the two nodes of edge (0, 1) swapped in P3 fail the full-cover cubic pin"""
    oracle.build(mutant=6)
    f, ref = FIELDS["x3"]
    tris = full_cover_square(2)
    H, xp = 0.5, (0.1, -0.05)
    rv, _ = ref(xp[0], xp[1], H * H * kernel_second_moment("wendland_c2"))
    v, _ = mesh_field_p("wendland_c2", H, xp, tris, 3, f, mutant=6)
    assert abs(v - rv) > 1e-6


def test_input_node_positions_match_the_oracle():
    """the input generator's node lattice (used to sample fields for the GPU path) is the
    oracle's"""
    from paper_2507_21686_gb300.workloads import field_node_positions
    rng = np.random.default_rng(45)
    tris = rng.normal(size=(20, 6))
    for order in (1, 2, 3):
        assert np.allclose(field_node_positions(tris, order), oracle.field_nodes(tris, order), atol=1e-15)
