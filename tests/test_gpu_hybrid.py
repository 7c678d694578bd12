"""Hybrid FP32 mode (quadrature for triangles away from the particle, inside the support or
small and across its edge; closed form otherwise) through the C-ABI against the FP64 oracle,
within the FP32 tolerance for every output."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300 import workloads as W
from tests.helpers import TOL_FP32, rel_err, scales

pytestmark = pytest.mark.gpu

KERNELS = ["wendland_c2", "wendland_c4", "wendland_c6", "cubic_spline"]


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


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check(ctx, w, kernel, deg, sample, seed=5):
    g, gr, mo = ctx.boundary_integrals(_t(w.particles), _t(w.triangles), kernel, w.H, deg, "fp32_hybrid")
    st = ctx.stats()
    g, gr = g.double().cpu().numpy(), gr.double().cpu().numpy()
    mo = mo.double().cpu().numpy() if mo is not None else np.zeros((len(g), 0))
    idx = np.random.default_rng(seed).choice(len(w.particles), sample, replace=False)
    sub = w.particles[idx]
    off, pt = oracle.cull(sub, w.triangles, w.H)
    og, ogr, omo, fl = oracle.particle_sums(kernel, w.H, sub, w.triangles, off, pt, deg)
    assert fl.sum() == 0
    got = np.concatenate([g[idx, None], gr[idx], mo[idx]], axis=1)
    ref = np.concatenate([og[:, None], ogr, omo], axis=1)
    err = rel_err(got, ref, scales(kernel, w.H, mo.shape[1]))
    return err.max(), st


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("deg", [-1, 1, 3])
def test_hybrid_box_vs_oracle(ctx, kernel, deg):
    w = W.box_obstacle(2, 128, 32)
    err, st = check(ctx, w, kernel, deg, 300)
    assert err <= TOL_FP32, err
    # a real share of the pairs took the quadrature (the rest the closed form)
    assert 0 < st["n_fallback"] < 0.9 * st["n_pairs"]


def triangle_soup(seed, n=24, count=2500, lo=0.05, hi=1.2):
    """jittered n x n particles in [0,1]^2 (H = 2.5/n) under overlapping generic triangles of
    longest edge ~ logU[lo, hi] H with centroids over [-H, 1+H]^2: every size class across
    the support edge, on both sides of each kernel's size limit for quadrature there"""
    rng = np.random.default_rng(seed)
    H = 2.5 / n
    parts = W.jittered_lattice(n, 1.0 / n, 0.25, rng)
    c = rng.uniform(-H, 1.0 + H, size=(count, 2))
    s = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)) * H * 0.5
    ang = rng.uniform(0, 2 * np.pi, size=(count, 1)) + np.array([0.0, 2.1, 4.2]) + rng.uniform(-0.5, 0.5, (count, 3))
    rad = s[:, None] * rng.uniform(0.6, 1.0, size=(count, 3))
    v = np.stack([c[:, None, 0] + rad * np.cos(ang), c[:, None, 1] + rad * np.sin(ang)], axis=-1)
    tris = v.reshape(count, 6).astype(np.float32)
    return W.Workload(f"triangle_soup_{n * n}_x_{count}", H, KERNELS, 3, parts, tris)


@pytest.mark.parametrize("kernel", KERNELS)
def test_hybrid_mixed_sizes_vs_oracle(ctx, kernel):
    w = triangle_soup(11)
    err, st = check(ctx, w, kernel, 3, 200)
    assert err <= TOL_FP32, err
    assert 0.05 * st["n_pairs"] < st["n_fallback"] < 0.95 * st["n_pairs"]


def test_hybrid_full_size_sampled(ctx):
    w = W.box_obstacle()
    err, st = check(ctx, w, "wendland_c4", 3, 150)
    assert err <= TOL_FP32, err
    print(f"\nhybrid C4 full size: closed form for {st['n_fallback'] / st['n_pairs']:.3f} of {st['n_pairs']} pairs")


def test_hybrid_deterministic_and_unsupported_paths(ctx):
    import torch
    from paper_2507_21686_gb300._lib import Sph2dError
    w = W.wall_strip()
    a = ctx.boundary_integrals(_t(w.particles), _t(w.triangles), "wendland_c2", w.H, 3, "fp32_hybrid")
    b = ctx.boundary_integrals(_t(w.particles), _t(w.triangles), "wendland_c2", w.H, 3, "fp32_hybrid")
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    pairs = np.zeros((4, 8))
    pairs[:, 2:] = [0.1, 0.1, 0.3, 0.1, 0.2, 0.3]
    with pytest.raises(Sph2dError, match="UNSUPPORTED"):
        ctx.pair_integrals(_t(pairs), "wendland_c2", 1.0, -1, "fp32_hybrid")
    with pytest.raises(Sph2dError, match="UNSUPPORTED"):
        ctx.backward(_t(w.particles), _t(w.triangles), "wendland_c2", w.H,
                     torch.zeros(len(w.particles), device="cuda"), "fp32_hybrid")


def cubic_near_pairs(seed, count, lmax_lo, lmax_hi):
    """one generic triangle per particle (particles 3 H apart, H = 1) that lies within H/2 of its
    particle but not inside r < H/2, innermost vertex inside r < H/2, at least 0.55 of its longest
    edge from the particle, longest edge in [lmax_lo, lmax_hi) H"""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        r0 = rng.uniform(0.05, 0.46)
        a0 = rng.uniform(0, 2 * np.pi)
        v0 = r0 * np.array([np.cos(a0), np.sin(a0)])
        L = rng.uniform(0.1, 0.5, 2)
        ang = a0 + rng.uniform(-1.4, 1.4, 2)
        v = np.stack([v0, v0 + L[0] * np.array([np.cos(ang[0]), np.sin(ang[0])]),
                      v0 + L[1] * np.array([np.cos(ang[1]), np.sin(ang[1])])])
        r = np.hypot(v[:, 0], v[:, 1])
        lmax = max(np.hypot(*(v[(i + 1) % 3] - v[i])) for i in range(3))
        d = _tri_dist(v)
        if (np.argmin(r) == 0 and r.max() > 0.52 and d < 0.48 and d >= 0.55 * lmax and lmax_lo <= lmax < lmax_hi
                and abs((v[1, 0] - v[0, 0]) * (v[2, 1] - v[0, 1]) - (v[1, 1] - v[0, 1]) * (v[2, 0] - v[0, 0])) > 1e-3):
            out.append(v)
    loc = np.array(out)
    n = int(np.ceil(np.sqrt(count)))
    centres = 3.0 * np.stack(np.meshgrid(np.arange(n), np.arange(n)), -1).reshape(-1, 2)[:count]
    parts = np.zeros((count, 4), dtype=np.float32)
    parts[:, :2] = centres
    tris = (loc + centres[:, None, :]).reshape(count, 6).astype(np.float32)
    return W.Workload(f"cubic_near_{count}", 1.0, ["cubic_spline"], 3, parts, tris)


def _tri_dist(v):
    """distance from the origin to the triangle v (3 x 2), 0 inside"""
    s = [(v[(e + 1) % 3, 0] - v[e, 0]) * (-v[e, 1]) - (v[(e + 1) % 3, 1] - v[e, 1]) * (-v[e, 0]) for e in range(3)]
    if all(x >= 0 for x in s) or all(x <= 0 for x in s):
        return 0.0
    best = np.inf
    for e in range(3):
        a, b = v[e], v[(e + 1) % 3]
        t = np.clip(-a @ (b - a) / ((b - a) @ (b - a)), 0.0, 1.0)
        best = min(best, np.hypot(*(a + t * (b - a))))
    return best


def test_hybrid_cubic_second_piece_by_quadrature(ctx):
    """cubic spline pairs within H/2 whose second piece the finer rule takes in the doubled frame
    (longest edge below 0.45 H): every pair by quadrature, each within 2e-6 of the output scales
    (the rule's 7.8e-7 in exact arithmetic plus FP32 rounding)"""
    w = cubic_near_pairs(31, 400, 0.1, 0.43)
    err, st = check(ctx, w, "cubic_spline", 3, 400)
    assert st["n_pairs"] == 400 and st["n_fallback"] == 0
    assert err <= 2e-6, err


def test_hybrid_cubic_near_large_to_closed_form(ctx):
    """the same class with longest edges of 0.46-0.5 H: beyond the finer rule's size, so the
    closed form takes them (within the FP32 tolerance)"""
    w = cubic_near_pairs(32, 200, 0.46, 0.5)
    err, st = check(ctx, w, "cubic_spline", 3, 200)
    assert st["n_pairs"] == 200 and st["n_fallback"] == 200
    assert err <= TOL_FP32, err
