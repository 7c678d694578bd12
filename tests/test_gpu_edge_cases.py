"""Edge cases of the widened entry points through the C-ABI: builds without particles, without
triangles or without any culled pair; zero-area and repeated-vertex triangles; a single pair.
Every output must be defined (zeros where nothing contributes) and agree with the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import pressure as OP
from paper_2507_21686_gb300.workloads import field_node_positions
from tests.helpers import TOL_FP32, TOL_FP64, rel_err, scales

pytestmark = pytest.mark.gpu


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


def parts_of(xy):
    p = np.zeros((len(xy), 4), dtype=np.float32)
    if len(xy):
        p[:, :2] = xy
    return p


CASES = {
    "no_particles": (np.zeros((0, 2)), np.array([[0.0, 0.0, 1.0, 0.0, 0.0, 1.0]])),
    "no_triangles": (np.array([[0.2, 0.2], [0.5, 0.5]]), np.zeros((0, 6))),
    "no_pairs": (np.array([[5.0, 5.0], [6.0, 5.5]]), np.array([[0.0, 0.0, 1.0, 0.0, 0.0, 1.0]])),
}


@pytest.mark.parametrize("case", list(CASES))
def test_empty_builds(ctx, case):
    import torch
    xy, tris = CASES[case]
    parts, tris = parts_of(xy), tris.astype(np.float32)
    N, M = len(parts), len(tris)
    H = 0.5
    ctx.build_cells(_t(parts), _t(tris), H)
    for mode in ("fp64", "fp32_fixup", "fp32_hybrid"):
        g, gr, mo = ctx.boundary_integrals(_t(parts), _t(tris), "wendland_c2", H, 3, mode)
        assert g.shape == (N,) and torch.count_nonzero(g) == 0 and torch.count_nonzero(gr) == 0
    for order, nn in ((1, 3), (2, 6), (3, 10)):
        vv = np.ones((M, nn, 2), dtype=np.float32)
        for mode in (("fp64", "fp32_fixup") if order == 1 else ("fp64", "fp32_hybrid")):
            v, gv = ctx.field_integrals(_t(vv), "wendland_c4", mode, order=order)
            assert v.shape == (N, 2) and torch.count_nonzero(v) == 0 and torch.count_nonzero(gv) == 0
    one = torch.ones(N, device="cuda")
    for model in (1, 2):
        a = ctx.boundary_pressure(one, one, one, 1000.0, "wendland_c2", "fp32_fixup", model)
        assert a.shape == (N, 2) and torch.count_nonzero(a) == 0
    q = ctx.mls_pressure(one, one, torch.zeros((0, 2), device="cuda"), "wendland_c2", "fp32_fixup")
    assert q.shape == (0,)
    if N == 0:
        q = ctx.mls_pressure(one, one, torch.zeros((3, 2), device="cuda"), "wendland_c2", "fp64")
        assert torch.count_nonzero(q) == 0                    # no particle within H of any point


def test_degenerate_triangles(ctx):
    """zero-area triangles (collinear, repeated vertex, all equal) contribute nothing in every
    mode and entry point; the one proper triangle matches the oracle"""
    parts = parts_of(np.array([[0.1, 0.05], [0.3, 0.2]]))
    good = [0.0, 0.0, 0.4, 0.0, 0.1, 0.3]
    tris = np.array([good,
                     [0.0, 0.1, 0.2, 0.1, 0.4, 0.1],      # collinear
                     [0.1, 0.1, 0.1, 0.1, 0.3, 0.2],      # repeated vertex
                     [0.2, 0.2, 0.2, 0.2, 0.2, 0.2]],     # a point
                    dtype=np.float32)
    H = 0.5
    ctx.build_cells(_t(parts), _t(tris), H)
    off, pt = oracle.cull(parts, tris[:1], H)
    og, ogr, omo, _ = oracle.particle_sums("cubic_spline", H, parts, tris[:1], off, pt, 3)
    ref = np.concatenate([og[:, None], ogr, omo], 1)
    for mode, tol in (("fp64", TOL_FP64), ("fp32_fixup", TOL_FP32), ("fp32_hybrid", TOL_FP32)):
        g, gr, mo = ctx.boundary_integrals(_t(parts), _t(tris), "cubic_spline", H, 3, mode)
        got = np.concatenate([g.double().cpu().numpy()[:, None], gr.double().cpu().numpy(),
                              mo.double().cpu().numpy()], 1)
        assert rel_err(got, ref, scales("cubic_spline", H, 10)).max() <= tol, mode
    # fields of order 2 and 3 on the same mesh: the degenerate triangles add nothing
    for order in (2, 3):
        nd = field_node_positions(tris, order)
        vv = (1.0 + nd[..., 0] - 2.0 * nd[..., 1] ** 2)[..., None].astype(np.float32)
        v, gv = ctx.field_integrals(_t(vv), "wendland_c2", "fp64", order=order)
        offo, pto = oracle.cull(parts, tris[:1], H)
        rv, rg = oracle.particle_field_sums_p("wendland_c2", H, parts, tris[:1], offo, pto, order, vv[:1])
        assert np.allclose(v.cpu().numpy(), rv, atol=1e-10)
        assert np.allclose(gv.cpu().numpy(), rg, atol=1e-9)
    # pressure model 2: contact points on a zero-area triangle still give finite values
    import torch
    rho = torch.full((2,), 1000.0, device="cuda")
    pr = torch.tensor([100.0, 200.0], device="cuda")
    vol = torch.full((2,), 0.01, device="cuda")
    for model in (1, 2):
        a = ctx.boundary_pressure(rho, pr, vol, 1000.0, "wendland_c2", "fp64", model).cpu().numpy()
        assert np.all(np.isfinite(a))
        offp, ptp = oracle.cull(parts, tris, H)
        ref = OP.boundary_pressure("wendland_c2", H, parts, tris, offp, ptp, rho.cpu().numpy(), pr.cpu().numpy(),
                                   vol.cpu().numpy(), 1000.0, model)
        assert np.allclose(a, ref, rtol=1e-9, atol=1e-12), (model, a, ref)


def test_single_pair_all_modes(ctx):
    """one particle and one triangle: every mode agrees with the oracle"""
    parts = parts_of(np.array([[0.05, -0.02]]))
    tris = np.array([[0.1, 0.1, 0.35, 0.05, 0.2, 0.4]], dtype=np.float32)
    H = 0.5
    off, pt = oracle.cull(parts, tris, H)
    for kernel in ("wendland_c2", "wendland_c6", "cubic_spline"):
        og, ogr, omo, _ = oracle.particle_sums(kernel, H, parts, tris, off, pt, 3)
        ref = np.concatenate([og[:, None], ogr, omo], 1)
        for mode, tol in (("fp64", TOL_FP64), ("fp32_fixup", TOL_FP32), ("fp32_hybrid", TOL_FP32)):
            g, gr, mo = ctx.boundary_integrals(_t(parts), _t(tris), kernel, H, 3, mode)
            got = np.concatenate([g.double().cpu().numpy()[:, None], gr.double().cpu().numpy(),
                                  mo.double().cpu().numpy()], 1)
            assert rel_err(got, ref, scales(kernel, H, 10)).max() <= tol, (kernel, mode)


def test_mls_after_builds_without_triangles(ctx):
    """MLS needs only the particles: after a build with no triangles (and after an unrelated
    build with another H before it) its grid must be this build's"""
    import torch
    rng = np.random.default_rng(71)
    xy = rng.uniform(0.0, 1.0, size=(2000, 2))
    parts = parts_of(xy)
    vol = np.full(len(xy), 1e-3, dtype=np.float32)
    p = (3.0 + xy[:, 0] - 2.0 * xy[:, 1]).astype(np.float32)
    pts = rng.uniform(0.1, 0.9, size=(50, 2)).astype(np.float32)
    other = parts_of(rng.uniform(0.0, 1.0, size=(100, 2)))
    ctx.build_cells(_t(other), _t(np.array([[0.0, 0.0, 1.0, 0.0, 0.0, 1.0]], dtype=np.float32)), 0.02)
    ctx.build_cells(_t(parts), _t(np.zeros((0, 6), dtype=np.float32)), 0.1)
    got = ctx.mls_pressure(_t(vol), _t(p), _t(pts), "wendland_c2", "fp64").cpu().numpy()
    ref = OP.mls_pressure("wendland_c2", 0.1, xy.astype(np.float32).astype(np.float64), vol.astype(np.float64),
                          p.astype(np.float64), pts.astype(np.float64))
    assert np.max(np.abs(got - ref)) < 1e-10 * np.abs(ref).max()


def test_fma_peak_measurement():
    """the FMA microbenchmark the bench reports against: plausible GB300 figures (derived FP32
    FMA peak 80.5 TFLOP/s; NVIDIA's FP64 figure 1.25 TFLOP/s) and argument checks"""
    import ctypes
    from paper_2507_21686_gb300 import _lib
    from paper_2507_21686_gb300.api import measure_fma_peak
    fp32 = measure_fma_peak(0, "fp32", 0.05)
    fp64 = measure_fma_peak(0, "fp64", 0.05)
    assert 40.0 < fp32 < 90.0, fp32
    assert 0.5 < fp64 < 2.0, fp64
    lib = _lib.load()
    out = ctypes.c_double()
    assert lib.sph2d_measure_fma_peak(0, 2, 0.05, ctypes.byref(out)) == 1
    assert lib.sph2d_measure_fma_peak(0, 0, 0.0, ctypes.byref(out)) == 1
    assert lib.sph2d_measure_fma_peak(0, 0, 0.05, None) == 1
