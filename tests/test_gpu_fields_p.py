"""Lagrange boundary fields of order 2 and 3 through the C-ABI against the oracle's polar
quadrature of the nodal field times W and grad W (a different route from the GPU's moments,
integration by parts and edge integrals, or its hybrid quadrature)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300 import workloads as W
from paper_2507_21686_gb300.workloads import field_node_positions, full_cover_square
from tests.helpers import TOL_FP32, TOL_FP64, scales

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


def smooth_node_values(tris, order, nf):
    """per-node samples of smooth fields of the world coordinates: [M, nodes, nf]"""
    v = field_node_positions(tris, order)
    x, y = v[..., 0], v[..., 1]
    fs = [np.sin(3 * x) + np.cos(2 * y) + 0.5 * x * y, 1.0 + x * x - 0.5 * y, 2.0 - x + 0.25 * y * y * y,
          np.exp(0.5 * x) * np.cos(y)]
    return np.stack(fs[:nf], axis=-1).astype(np.float32)


def field_err(got_v, got_g, ref_v, ref_g, vv, kernel, H):
    """errors relative to max(|ref|, field scale x output scale)"""
    A = np.max(np.abs(vv), axis=(0, 1))
    sc = scales(kernel, H, 0)
    ev = np.abs(got_v - ref_v) / np.maximum(np.abs(ref_v), A[None, :] * sc[0])
    eg = np.abs(got_g - ref_g) / np.maximum(np.abs(ref_g), A[None, :, None] * sc[1])
    return max(ev.max(), eg.max())


def check(ctx, w, kernel, order, mode, nf=3, sample=200, seed=7):
    parts, tris, H = w.particles, w.triangles, w.H
    vv = smooth_node_values(tris, order, nf)
    ctx.build_cells(_t(parts), _t(tris), H)
    val, gr = ctx.field_integrals(_t(vv), kernel, mode, order=order)
    st = ctx.stats()
    val, gr = val.double().cpu().numpy(), gr.double().cpu().numpy()
    idx = np.random.default_rng(seed).choice(len(parts), sample, replace=False)
    off, pt = oracle.cull(parts[idx], tris, H)
    rv, rg = oracle.particle_field_sums_p(kernel, H, parts[idx], tris, off, pt, order, vv)
    return field_err(val[idx], gr[idx], rv, rg, vv, kernel, H), st


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("mode", ["fp64", "fp32_hybrid"])
def test_fields_p_box_vs_oracle(ctx, kernel, order, mode):
    w = W.box_obstacle(2, 96, 24)
    err, st = check(ctx, w, kernel, order, mode)
    assert err <= (TOL_FP64 if mode == "fp64" else TOL_FP32), err
    if mode == "fp32_hybrid":
        assert 0 < st["n_fallback"] < 0.5 * st["n_pairs"]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("order", [2, 3])
def test_fields_p_triangle_soup_hybrid(ctx, kernel, order):
    """overlapping generic triangles of every size class (0.05-1.2 H) in the hybrid mode"""
    from tests.test_gpu_hybrid import triangle_soup
    err, st = check(ctx, triangle_soup(11), kernel, order, "fp32_hybrid", nf=2, sample=150)
    assert err <= TOL_FP32, err


@pytest.mark.parametrize("mode", ["fp64", "fp32_hybrid"])
def test_full_cover_cubic_field(ctx, mode):
    """support inside the 8-triangle [-1,1]^2 mesh (Sec. 6.2's full cover): f = x^3 gives
    <f> = x^3 + 3 x H^2 m2 and <grad f> = (3 (x^2 + H^2 m2), 0); f = x y gives x y and (y, x)"""
    from tests.test_oracle_field_p_pins import kernel_second_moment
    tris = full_cover_square(2).astype(np.float32)
    parts = np.array([[0.0, 0.0, 0.0, 0.0], [0.1, -0.05, 0.0, 0.0]], dtype=np.float32)
    nd = field_node_positions(tris, 3)
    vv = np.stack([nd[..., 0] ** 3, nd[..., 0] * nd[..., 1]], axis=-1).astype(np.float32)
    H = 0.5
    ctx.build_cells(_t(parts), _t(tris), H)
    val, gr = ctx.field_integrals(_t(vv), "wendland_c4", mode, order=3)
    val, gr = val.double().cpu().numpy(), gr.double().cpu().numpy()
    s = H * H * kernel_second_moment("wendland_c4")
    # the node values are float32 (the fields at nodes such as (1/3, -1/3) round by ~6e-8), so
    # the interpolated field is the polynomial only to that level
    tol = 3e-7 if mode == "fp64" else 1e-5
    for i in range(2):
        x, y = float(parts[i, 0]), float(parts[i, 1])
        assert abs(val[i, 0] - (x ** 3 + 3 * x * s)) < tol
        assert np.allclose(gr[i, 0], [3 * (x * x + s), 0.0], atol=tol * 10)
        assert abs(val[i, 1] - x * y) < tol
        assert np.allclose(gr[i, 1], [y, x], atol=tol * 10)


def test_linear_nodes_match_order_one(ctx):
    """a linear field sampled at P2 and P3 nodes gives the piecewise-linear result (to the
    float32 rounding of the node values, ~1e-7 of the field)"""
    w = W.wall_strip()
    parts, tris, H = w.particles, w.triangles, w.H
    ctx.build_cells(_t(parts), _t(tris), H)
    lin = lambda p: 1.0 + 2.0 * p[..., 0] - 0.5 * p[..., 1]
    v1, g1 = ctx.field_integrals(_t(lin(field_node_positions(tris, 1))[..., None].astype(np.float32)),
                                 "wendland_c2", "fp64")
    for order in (2, 3):
        vk, gk = ctx.field_integrals(_t(lin(field_node_positions(tris, order))[..., None].astype(np.float32)),
                                     "wendland_c2", "fp64", order=order)
        assert np.max(np.abs(vk.cpu().numpy() - v1.cpu().numpy())) < 1e-6
        assert np.max(np.abs(gk.cpu().numpy() - g1.cpu().numpy())) < 1e-6 / H


def test_fields_p_options_and_errors(ctx):
    import torch
    from paper_2507_21686_gb300._lib import Sph2dError
    w = W.wall_strip()
    parts, tris, H = w.particles, w.triangles, w.H
    ctx.build_cells(_t(parts), _t(tris), H)
    vv = smooth_node_values(tris, 3, 4)
    v4, g4 = ctx.field_integrals(_t(vv), "cubic_spline", "fp32_hybrid", order=3)
    for nf in (1, 2):
        v, g = ctx.field_integrals(_t(np.ascontiguousarray(vv[:, :, :nf])), "cubic_spline", "fp32_hybrid", order=3)
        assert torch.equal(v, v4[:, :nf]) and torch.equal(g, g4[:, :nf])
    v0, g0 = ctx.field_integrals(_t(vv), "cubic_spline", "fp32_hybrid", want_grad=False, order=3)
    assert g0 is None and torch.equal(v0, v4)
    v2, g2 = ctx.field_integrals(_t(vv), "cubic_spline", "fp32_hybrid", order=3)
    assert torch.equal(v2, v4) and torch.equal(g2, g4)          # deterministic
    with pytest.raises(Sph2dError, match="UNSUPPORTED"):
        ctx.field_integrals(_t(vv), "wendland_c2", "fp32_fixup", order=3)
    from paper_2507_21686_gb300._lib import check as check_status
    from paper_2507_21686_gb300.api import _ptr
    out = torch.empty((len(parts), 1), dtype=torch.float64, device="cuda")
    vt = _t(vv)
    with pytest.raises(Sph2dError, match="INVALID_ARG"):
        check_status(ctx.lib, ctx.h, ctx.lib.sph2d_field_integrals_p(ctx.h, 0, 0, 4, _ptr(vt), 1, _ptr(out), None))
    with pytest.raises(ValueError):
        ctx.field_integrals(_t(vv), "wendland_c2", "fp64", order=2)   # 10 nodes given, 6 expected
