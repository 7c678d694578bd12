"""The cubic spline's per-particle path treats the pairs within H/2 of their triangle (both
pieces of k = 2 (1-q)^3_+ - (1-2q)^3_+) apart from the others (first piece only): its batch
kernel gathers the near pairs of several 32-pair chunks into warp-wide rounds of second pieces
and adds each near pair's second piece to its first.  These cases put the boundaries where they
can go wrong: every pair near (one chunk per batch), every pair far (no second-piece round), a
pair count that is an exact multiple of the 32-pair chunk, near and far pairs that alternate
particle by particle, a particle whose near and far pairs each span several chunks, and chunks
whose near pairs exactly fill a round, overflow it by one or leave one lane.  Expected values
come from the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.test_gpu_parity import compare_particles

pytestmark = pytest.mark.gpu

TRI = np.array([[-0.2, -0.2, 0.3, -0.1, 0.0, 0.3]])
CENTROID = TRI.reshape(3, 2).mean(axis=0)


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2507_21686_gb300 import build
    build.build()
    from paper_2507_21686_gb300.api import Context
    c = Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def parts_of(xy):
    p = np.zeros((len(xy), 4), dtype=np.float32)
    p[:, :2] = xy
    return p


def ring(rng, n, r0, r1):
    """n points at distance [r0, r1) from the triangle's centroid"""
    r = rng.uniform(r0, r1, n)
    a = rng.uniform(0.0, 2.0 * np.pi, n)
    return CENTROID + np.stack([r * np.cos(a), r * np.sin(a)], axis=1)


def polar_mesh(radius, n_ring, n_seg):
    """a disk of radius `radius` around the origin in triangles: a central fan and quads split in
    two, about radius / n_ring across"""
    rs = radius * np.arange(n_ring + 1) / n_ring
    th = 2.0 * np.pi * np.arange(n_seg + 1) / n_seg
    P = lambda r, t: (r * np.cos(t), r * np.sin(t))
    tris = []
    for j in range(n_seg):
        tris.append([0.0, 0.0, *P(rs[1], th[j]), *P(rs[1], th[j + 1])])
    for k in range(1, n_ring):
        for j in range(n_seg):
            a, b = P(rs[k], th[j]), P(rs[k], th[j + 1])
            c, d = P(rs[k + 1], th[j]), P(rs[k + 1], th[j + 1])
            tris.append([*a, *c, *d])
            tris.append([*a, *d, *b])
    return np.array(tris)


def check_parts(parts, tris, H, expect_near, expect_far):
    """the oracle's cull gives the expected numbers of near (distance < H/2) and far pairs"""
    off, pt = oracle.cull(parts, tris, H)
    near = 0
    for i in range(len(parts)):
        for t in pt[off[i]:off[i + 1]]:
            v = tris[t].reshape(3, 2).astype(np.float64) - parts[i, :2].astype(np.float64)
            near += seg_tri_dist(v) < 0.5 * H
    far = len(pt) - near
    if expect_near is not None:
        assert near == expect_near
    if expect_far is not None:
        assert far == expect_far
    return near, far


def seg_tri_dist(v):
    """distance from the origin to the triangle with vertices v (3 x 2)"""
    s = []
    for e in range(3):
        a, b = v[e], v[(e + 1) % 3]
        s.append((b[0] - a[0]) * (-a[1]) - (b[1] - a[1]) * (-a[0]))
    if all(x >= 0 for x in s) or all(x <= 0 for x in s):
        return 0.0
    best = np.inf
    for e in range(3):
        a, b = v[e], v[(e + 1) % 3]
        ab = b - a
        t = np.clip(-a @ ab / (ab @ ab), 0.0, 1.0)
        best = min(best, np.hypot(*(a + t * ab)))
    return best


MODES = ["fp32_fixup", "fp64"]


@pytest.mark.parametrize("mode", MODES)
def test_all_pairs_near(ctx, mode):
    """64 particles within 0.4 H of the centroid of one triangle: every pair near, P = 64"""
    rng = np.random.default_rng(91)
    parts = parts_of(ring(rng, 64, 0.0, 0.4))
    check_parts(parts, TRI, 1.0, 64, 0)
    compare_particles(ctx, parts, TRI.astype(np.float32), 1.0, "cubic_spline", 3, mode)


@pytest.mark.parametrize("mode", MODES)
def test_all_pairs_far(ctx, mode):
    """64 particles 0.95-1.0 H from the centroid: every pair between H/2 and H, P = 64"""
    rng = np.random.default_rng(92)
    parts = parts_of(ring(rng, 64, 0.95, 1.0))
    check_parts(parts, TRI, 1.0, 0, 64)
    compare_particles(ctx, parts, TRI.astype(np.float32), 1.0, "cubic_spline", 3, mode)


@pytest.mark.parametrize("mode", MODES)
def test_alternating_near_and_far(ctx, mode):
    """particles alternate near / far / without pairs: every chunk holds both parts"""
    rng = np.random.default_rng(93)
    near, far, none = ring(rng, 40, 0.0, 0.4), ring(rng, 40, 0.95, 1.0), ring(rng, 20, 3.0, 4.0)
    xy = np.empty((100, 2))             # near, far, near, far, none, near, ...
    xy[0::5], xy[1::5], xy[2::5], xy[3::5], xy[4::5] = near[:20], far[:20], near[20:], far[20:], none
    parts = parts_of(xy)
    check_parts(parts, TRI, 1.0, 40, 40)
    compare_particles(ctx, parts, TRI.astype(np.float32), 1.0, "cubic_spline", 3, mode)


@pytest.mark.parametrize("mode", MODES)
def test_parts_spanning_chunks(ctx, mode):
    """a fine polar mesh: the particle at its centre has ~200 near and ~200 far pairs, each part
    over several chunks; other particles inside, on and beyond the mesh's rim"""
    tris = polar_mesh(1.6, 13, 24).astype(np.float32)
    rng = np.random.default_rng(94)
    xy = np.concatenate([[[0.0, 0.0]], rng.uniform(-1.2, 1.2, size=(30, 2)),
                         [[1.6, 0.0], [0.0, -1.65], [2.4, 2.4]]])
    parts = parts_of(xy)
    near, far = check_parts(parts[:1], tris, 1.0, None, None)
    assert near > 64 and far > 64
    compare_particles(ctx, parts, tris, 1.0, "cubic_spline", 3, mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("per_chunk", [16, 17, 31])
def test_near_pairs_filling_the_second_piece_rounds(ctx, mode, per_chunk):
    """chunks of 32 pairs with a fixed number of near pairs each, so that the near pairs of two
    chunks exactly fill one warp-wide round of second pieces (16), overflow it by one pair and
    start the next batch (17), or leave one lane (31); 12 chunks, one pair per particle"""
    rng = np.random.default_rng(95 + per_chunk)
    xy = []
    for _ in range(12):
        near, far = ring(rng, per_chunk, 0.0, 0.4), ring(rng, 32 - per_chunk, 0.95, 1.0)
        chunk = np.concatenate([near, far])
        xy.append(chunk[rng.permutation(32)])
    parts = parts_of(np.concatenate(xy))
    check_parts(parts, TRI, 1.0, 12 * per_chunk, 12 * (32 - per_chunk))
    compare_particles(ctx, parts, TRI.astype(np.float32), 1.0, "cubic_spline", 3, mode)
