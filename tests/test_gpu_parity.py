"""GPU path vs the FP64 oracle through the C-ABI: bit-exact pair lists, per-particle and
per-pair integrals within the stated tolerances, edge cases and error statuses."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300 import workloads as W
from tests.helpers import TOL_FP32, TOL_FP64, oracle_per_pair, pair_rel_err, rel_err, scales

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


def _t(a, dev="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def gpu_pairs(ctx, parts, tris, H):
    ctx.build_cells(_t(parts), _t(tris), H)
    off, tri = ctx.pair_list()
    return off.cpu().numpy(), tri.cpu().numpy()


def compare_particles(ctx, parts, tris, H, kernel, deg, mode, sample=None, tol=None):
    """Full GPU path vs oracle per-particle sums (optionally on a particle sample)."""
    g, gr, mo = ctx.boundary_integrals(_t(parts), _t(tris), kernel, H, deg, mode)
    g, gr = g.cpu().numpy(), gr.cpu().numpy()
    mo = mo.cpu().numpy() if mo is not None else np.zeros((len(parts), 0))
    idx = np.arange(len(parts)) if sample is None else sample
    sub = parts[idx]
    off, pt = oracle.cull(sub, tris, H)
    og, ogr, omo, fl = oracle.particle_sums(kernel, H, sub, tris, off, pt, deg)
    assert fl.sum() == 0
    nm = mo.shape[1]
    got = np.concatenate([g[idx, None], gr[idx], mo[idx]], axis=1)
    ref = np.concatenate([og[:, None], ogr, omo], axis=1)
    err = rel_err(got, ref, scales(kernel, H, nm))
    tol = tol if tol is not None else (TOL_FP64 if mode == "fp64" else TOL_FP32)
    worst = np.unravel_index(np.argmax(err), err.shape)
    assert err.max() <= tol, f"{kernel} {mode}: max err {err.max():.3e} at particle {idx[worst[0]]} output {worst[1]}"
    return err.max()


# ---------------------------------------------------------------------------------------
# culling
# ---------------------------------------------------------------------------------------
def test_cull_bit_exact_wall_strip(ctx):
    w = W.wall_strip()
    off, tri = gpu_pairs(ctx, w.particles, w.triangles, w.H)
    roff, rtri = oracle.cull(w.particles, w.triangles, w.H)
    assert np.array_equal(off, roff)
    assert np.array_equal(tri, rtri)
    assert len(tri) > 500


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cull_bit_exact_random_mixed_sizes(ctx, seed):
    rng = np.random.default_rng(100 + seed)
    n, m = 3001, 517                                  # ragged sizes
    parts = np.zeros((n, 4), np.float32)
    parts[:, :2] = rng.uniform(-0.2, 1.2, size=(n, 2))
    c = rng.uniform(0, 1, size=(m, 2))
    size = np.exp(rng.uniform(np.log(0.002), np.log(0.6), size=m))
    tris = (np.repeat(c, 3, axis=0).reshape(m, 6) + rng.uniform(-1, 1, size=(m, 6)) * size[:, None])
    tris = tris.astype(np.float32)
    H = 0.03
    off, tri = gpu_pairs(ctx, parts, tris, H)
    roff, rtri = oracle.cull(parts, tris, H)
    assert np.array_equal(off, roff)
    assert np.array_equal(tri, rtri)


def test_cull_threshold_cases(ctx):
    """Particles placed at distance ~H (ties decided by the FP64 predicate) and on edges."""
    H = 0.125
    tris = np.array([[0, 0, 1, 0, 0, 1], [2, 2, 3, 2, 2.5, 3], [0.5, -1, 0.5, -1, 0.5, -0.5]],
                    np.float32)
    pts = []
    for d in [H * (1 - 1e-7), H, H * (1 + 1e-7), 0.0, 1e-30]:
        pts += [[0.3, -d], [-d, 0.3], [0.5 + d * 0.70710678, 0.5 + d * 0.70710678], [2.5, 2 - d]]
    pts += [[0.0, 0.0], [1.0, 0.0], [0.5, -0.75]]
    parts = np.zeros((len(pts), 4), np.float32)
    parts[:, :2] = np.array(pts, np.float32)
    off, tri = gpu_pairs(ctx, parts, tris, H)
    roff, rtri = oracle.cull(parts, tris, H)
    assert np.array_equal(off, roff) and np.array_equal(tri, rtri)


def test_cull_empty_inputs(ctx):
    import torch
    parts = np.zeros((5, 4), np.float32)
    tris = np.zeros((0, 6), np.float32)
    off, tri = gpu_pairs(ctx, parts, tris, 0.1)
    assert np.all(off == 0) and len(tri) == 0
    g, gr, _ = ctx.boundary_integrals(_t(parts), _t(tris), "wendland_c2", 0.1)
    assert torch.all(g == 0) and torch.all(gr == 0)
    g, gr, _ = ctx.boundary_integrals(_t(np.zeros((0, 4), np.float32)),
                                      _t(np.ones((3, 6), np.float32)), "wendland_c2", 0.1)
    assert g.numel() == 0


def test_cull_full_size_sampled(ctx):
    w = W.box_obstacle()
    off, tri = gpu_pairs(ctx, w.particles, w.triangles, w.H)
    rng = np.random.default_rng(7)
    near = np.nonzero(np.diff(off) > 0)[0]
    sample = np.sort(np.concatenate([rng.choice(len(w.particles), 200, replace=False),
                                     rng.choice(near, 300, replace=False)]))
    roff, rtri = oracle.cull(w.particles[sample], w.triangles, w.H)
    for k, i in enumerate(sample):
        assert np.array_equal(tri[off[i]:off[i + 1]], rtri[roff[k]:roff[k + 1]]), f"particle {i}"


# ---------------------------------------------------------------------------------------
# per-particle integrals
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["fp64", "fp32_fixup"])
@pytest.mark.parametrize("kernel", KERNELS)
def test_wall_strip_all_outputs(ctx, kernel, mode):
    w = W.wall_strip()
    compare_particles(ctx, w.particles, w.triangles, w.H, kernel, 3, mode)


@pytest.mark.parametrize("kernel", ["wendland_c4", "cubic_spline"])
@pytest.mark.parametrize("deg", [-1, 0, 1, 2])
def test_moment_degrees(ctx, deg, kernel):
    """every moment-degree instance (none, first moments, all ten) of a single-polynomial kernel
    and of the cubic spline's batch kernel"""
    w = W.wall_strip()
    for mode in ("fp64", "fp32_fixup"):
        compare_particles(ctx, w.particles, w.triangles, w.H, kernel, deg, mode)


@pytest.mark.parametrize("mode", ["fp64", "fp32_fixup"])
@pytest.mark.parametrize("kernel", ["wendland_c2", "cubic_spline"])
def test_box_obstacle_small_full(ctx, kernel, mode):
    w = W.box_obstacle(n=128)
    compare_particles(ctx, w.particles, w.triangles, w.H, kernel, 3, mode)


@pytest.mark.parametrize("mode", ["fp64", "fp32_fixup"])
@pytest.mark.parametrize("kernel", ["wendland_c2", "wendland_c4", "cubic_spline"])
def test_box_obstacle_full_size_sampled(ctx, kernel, mode):
    """Full-size workload in the benchmark's launch configuration, oracle on a sample."""
    w = W.box_obstacle()
    off, _ = gpu_pairs(ctx, w.particles, w.triangles, w.H)
    rng = np.random.default_rng(8)
    near = np.nonzero(np.diff(off) > 0)[0]
    sample = np.sort(np.concatenate([rng.choice(len(w.particles), 64, replace=False),
                                     rng.choice(near, 192, replace=False)]))
    compare_particles(ctx, w.particles, w.triangles, w.H, kernel, 3, mode, sample=sample)


def test_paper_full_cover_and_wall(ctx):
    """Sec. 6.2: [-1,1]^2 in 8 triangles, x = 0, h = 1 -> gamma = 1, grad = 0; and a particle
    on a straight wall -> gamma = 1/2."""
    import torch
    tris = W.full_cover_square(2).astype(np.float32)
    parts = np.zeros((2, 4), np.float32)
    parts[1, :2] = [0.0, -1.0]                       # on the bottom wall of the square
    for mode, tol in (("fp64", TOL_FP64), ("fp32_fixup", TOL_FP32)):
        for k in KERNELS:
            g, gr, _ = ctx.boundary_integrals(_t(parts), _t(tris), k, 1.0, -1, mode)
            g, gr = g.cpu().double().numpy(), gr.cpu().double().numpy()
            sg = scales(k, 1.0, 0)[1]
            assert abs(g[0] - 1.0) <= tol and np.all(np.abs(gr[0]) <= tol * sg)
            assert abs(g[1] - 0.5) <= tol
    del torch


# ---------------------------------------------------------------------------------------
# independent pairs (precision stress)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", KERNELS)
def test_stress_pairs_per_pair(ctx, kernel):
    w = W.precision_stress(count=6000)
    pairs = w.pairs
    ref = oracle_per_pair(oracle.pairs(kernel, 1.0, pairs), 10)
    sc = scales(kernel, 1.0, 10)
    for mode, tol in (("fp64", TOL_FP64), ("fp32_fixup", TOL_FP32)):
        out = ctx.pair_integrals(_t(pairs), kernel, 1.0, 3, mode).cpu().numpy()
        err = rel_err(out, ref, sc)
        for c in range(3):
            e = err[w.labels == c].max()
            assert e <= tol, f"{kernel} {mode} class {c}: {e:.3e}"


def test_stress_pairs_world_units(ctx):
    """Per-pair entry with H != 1 and particles away from the origin."""
    rng = np.random.default_rng(21)
    w = W.precision_stress(count=900)
    H = 0.0371
    shift = rng.uniform(-3, 3, size=(len(w.pairs), 2))
    pairs = w.pairs * H
    pairs[:, 0::2] += shift[:, :1]
    pairs[:, 1::2] += shift[:, 1:]
    ref = oracle_per_pair(oracle.pairs("wendland_c2", H, pairs), 10)
    out = ctx.pair_integrals(_t(pairs), "wendland_c2", H, 3, "fp64").cpu().numpy()
    assert rel_err(out, ref, scales("wendland_c2", H, 10)).max() <= TOL_FP64


def test_huge_triangles_take_the_fixup_path(ctx):
    pairs = np.zeros((64, 8))
    rng = np.random.default_rng(22)
    pairs[:, 2:] = rng.uniform(-60, 60, size=(64, 6))
    pairs[:, 2:4] = rng.uniform(-0.5, 0.5, size=(64, 2))      # one vertex near the particle
    ref = oracle_per_pair(oracle.pairs("wendland_c4", 1.0, pairs), 10)
    out = ctx.pair_integrals(_t(pairs), "wendland_c4", 1.0, 3, "fp32_fixup").cpu().numpy()
    assert rel_err(out, ref, scales("wendland_c4", 1.0, 10)).max() <= TOL_FP32
    assert ctx.stats()["n_fixup"] > 0


@pytest.mark.parametrize("kernel", ["wendland_c2", "cubic_spline"])
@pytest.mark.parametrize("mode", ["fp32_fixup", "fp32_hybrid"])
def test_huge_triangles_fixup_per_particle(ctx, kernel, mode):
    """per-particle path with triangles reaching 60 H: their FP32 local coordinates leave the
    trusted range, so those pairs take the FP64 fix-up (for the cubic spline, its own fix-up
    pass over a list)"""
    rng = np.random.default_rng(23)
    parts = np.zeros((32, 4), dtype=np.float32)
    parts[:, :2] = rng.uniform(-0.5, 0.5, size=(32, 2))
    tris = rng.uniform(-60, 60, size=(24, 6))
    tris[:, 0:2] = rng.uniform(-0.6, 0.6, size=(24, 2))       # one vertex among the particles
    tris = np.concatenate([tris, W.wall_strip().triangles[:8] * 4 - 1.5]).astype(np.float32)
    g, gr, mo = ctx.boundary_integrals(_t(parts), _t(tris), kernel, 1.0, 3, mode)
    st = ctx.stats()
    off, pt = oracle.cull(parts, tris, 1.0)
    og, ogr, omo, fl = oracle.particle_sums(kernel, 1.0, parts, tris, off, pt, 3)
    got = np.concatenate([g.double().cpu().numpy()[:, None], gr.double().cpu().numpy(), mo.double().cpu().numpy()], 1)
    ref = np.concatenate([og[:, None], ogr, omo], 1)
    assert rel_err(got, ref, scales(kernel, 1.0, 10)).max() <= TOL_FP32
    assert st["n_fixup"] > 0


# ---------------------------------------------------------------------------------------
# behaviour
# ---------------------------------------------------------------------------------------
def test_orientation_and_degenerate_triangles(ctx):
    w = W.wall_strip()
    cw = w.triangles.reshape(-1, 3, 2)[:, [0, 2, 1]].reshape(-1, 6).copy()
    a = ctx.boundary_integrals(_t(w.particles), _t(w.triangles), "wendland_c2", w.H, 3, "fp64")
    b = ctx.boundary_integrals(_t(w.particles), _t(cw), "wendland_c2", w.H, 3, "fp64")
    sc = scales("wendland_c2", w.H, 10)
    ga = np.concatenate([a[0].cpu().numpy()[:, None], a[1].cpu().numpy(), a[2].cpu().numpy()], 1)
    gb = np.concatenate([b[0].cpu().numpy()[:, None], b[1].cpu().numpy(), b[2].cpu().numpy()], 1)
    assert rel_err(ga, gb, sc).max() <= 1e-13
    deg = np.array([[0.1, 0.0, 0.2, 0.0, 0.3, 0.0], [0.1, 0.01, 0.1, 0.01, 0.2, 0.02]], np.float32)
    parts = np.zeros((3, 4), np.float32)
    parts[:, :2] = [[0.15, 0.0], [0.15, 0.05], [0.1, 0.01]]
    for mode in ("fp64", "fp32_fixup"):
        g, gr, mo = ctx.boundary_integrals(_t(parts), _t(deg), "wendland_c2", 0.125, 3, mode)
        assert np.all(g.cpu().numpy() == 0) and np.all(gr.cpu().numpy() == 0)
        assert np.all(mo.cpu().numpy() == 0)


@pytest.mark.parametrize("kernel", ["wendland_c2", "cubic_spline"])
def test_deterministic_bitwise(ctx, kernel):
    """repeated calls give identical bits (dynamic chunk scheduling; for the cubic spline also
    its near/far partition)"""
    w = W.box_obstacle(n=128)
    r = [ctx.boundary_integrals(_t(w.particles), _t(w.triangles), kernel, w.H, 3, m)
         for m in ("fp32_fixup", "fp32_fixup", "fp64", "fp64")]
    for i in (0, 2):
        for x, y in zip(r[i], r[i + 1]):
            assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_integrals_from_pairs_reuses_the_cull(ctx):
    w = W.wall_strip()
    a = ctx.boundary_integrals(_t(w.particles), _t(w.triangles), "wendland_c4", w.H, 3, "fp64")
    b = ctx.integrals_from_pairs("wendland_c4", 3, "fp64")
    for x, y in zip(a, b):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_error_statuses(ctx):
    import torch
    from paper_2507_21686_gb300._lib import Sph2dError
    w = W.wall_strip()
    bad = w.particles.copy()
    bad[5, 0] = np.nan
    with pytest.raises(Sph2dError) as e:
        ctx.boundary_integrals(_t(bad), _t(w.triangles), "wendland_c2", w.H)
    assert e.value.status == 2
    badt = w.triangles.copy()
    badt[3, 4] = np.inf
    with pytest.raises(Sph2dError) as e:
        ctx.boundary_integrals(_t(w.particles), _t(badt), "wendland_c2", w.H)
    assert e.value.status == 2
    for H in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(Sph2dError) as e:
            ctx.boundary_integrals(_t(w.particles), _t(w.triangles), "wendland_c2", H)
        assert e.value.status == 1
    with pytest.raises(Sph2dError) as e:
        ctx.boundary_integrals(_t(w.particles), _t(w.triangles), 7, w.H)
    assert e.value.status == 1
    with pytest.raises(Sph2dError) as e:
        ctx.boundary_integrals(_t(w.particles), _t(w.triangles), "wendland_c2", w.H, 4)
    assert e.value.status == 1
    # the context stays usable after errors
    g, _, _ = ctx.boundary_integrals(_t(w.particles), _t(w.triangles), "wendland_c2", w.H)
    assert torch.isfinite(g).all()


def test_pair_list_capacity_status(ctx):
    import ctypes
    import torch
    from paper_2507_21686_gb300.api import _ptr
    w = W.wall_strip()
    ctx.build_cells(_t(w.particles), _t(w.triangles), w.H)
    P = ctx.pair_count()
    off = torch.empty(len(w.particles) + 1, dtype=torch.int64, device="cuda")
    tri = torch.empty(P, dtype=torch.int32, device="cuda")
    req = ctypes.c_int64()
    st = ctx.lib.sph2d_pair_list(ctx.h, _ptr(off), _ptr(tri), P - 1, ctypes.byref(req))
    assert st == 3 and req.value == P


@pytest.mark.parametrize("kernel", ["wendland_c2", "wendland_c4", "wendland_c6"])
def test_stress_pairs_full_size(ctx, kernel):
    """All 262,144 precision-stress pairs (generic / sliver / near-singular), every output."""
    w = W.precision_stress()
    ref = oracle_per_pair(oracle.pairs(kernel, 1.0, w.pairs), 10)
    sc = scales(kernel, 1.0, 10)
    for mode, tol in (("fp64", TOL_FP64), ("fp32_fixup", TOL_FP32)):
        out = ctx.pair_integrals(_t(w.pairs), kernel, 1.0, 3, mode).cpu().numpy()
        err = rel_err(out, ref, sc).max(axis=1)
        for c in range(3):
            assert err[w.labels == c].max() <= tol, f"{kernel} {mode} class {c}: {err[w.labels == c].max():.3e}"
        # relative to each pair's own value, down to 1e-6 of the output scale: a 1e-3 H triangle
        # or a sliver has gamma ~ 1e-6, where the fan decomposition's cancellation leaves the FP64
        # path an absolute error of about 1e-12 of the scale (bounded here) and FP32 rounding of
        # the local geometry alone moves the value by up to ~1e-1 of itself (reported only)
        ep = pair_rel_err(out, ref, sc).max(axis=1)
        print(f"\n{kernel} {mode} per-pair relative error (floor 1e-6 S_r), classes generic / sliver / "
              f"near-singular: " + " / ".join(f"{ep[w.labels == c].max():.1e}" for c in range(3)))
        if mode == "fp64":
            ea = (np.abs(out - ref) / sc).max()
            assert ea <= 3e-12, f"{kernel} fp64 absolute error {ea:.3e} of the scale"
