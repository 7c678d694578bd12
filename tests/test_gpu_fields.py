"""Piecewise-linear boundary fields through the C-ABI against the oracle's polar quadrature of
A W and A grad W (a different route from the GPU's moments + integration by parts)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300 import workloads as W
from paper_2507_21686_gb300.workloads import full_cover_square
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


def smooth_fields(tris, nf):
    """per-vertex samples of smooth fields of the world coordinates: [M, 3, nf]"""
    v = tris.reshape(-1, 3, 2).astype(np.float64)
    x, y = v[..., 0], v[..., 1]
    fs = [np.sin(3 * x) + np.cos(2 * y) + 0.5 * x * y, 1.0 + 0.0 * x, 2.0 - x + 0.25 * y, x * x - y]
    return np.stack(fs[:nf], axis=-1).astype(np.float32)


def field_err(got_v, got_g, ref_v, ref_g, vv, kernel, H):
    """errors relative to max(|ref|, field scale x output scale)"""
    A = np.max(np.abs(vv), axis=(0, 1))                        # per field
    sc = scales(kernel, H, 0)
    ev = np.abs(got_v - ref_v) / np.maximum(np.abs(ref_v), A[None, :] * sc[0])
    eg = np.abs(got_g - ref_g) / np.maximum(np.abs(ref_g), A[None, :, None] * sc[1])
    return max(ev.max(), eg.max())


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("mode", ["fp64", "fp32_fixup"])
def test_fields_box_vs_oracle(ctx, kernel, mode):
    w = W.box_obstacle(2, 96, 24)
    parts, tris, H = w.particles, w.triangles, w.H
    vv = smooth_fields(tris, 4)
    ctx.build_cells(_t(parts), _t(tris), H)
    val, gr = ctx.field_integrals(_t(vv), kernel, mode)
    val, gr = val.double().cpu().numpy(), gr.double().cpu().numpy()
    idx = np.random.default_rng(7).choice(len(parts), 250, replace=False)
    off, pt = oracle.cull(parts[idx], tris, H)
    rv, rg = oracle.particle_field_sums(kernel, H, parts[idx], tris, off, pt, vv)
    tol = TOL_FP64 if mode == "fp64" else TOL_FP32
    err = field_err(val[idx], gr[idx], rv, rg, vv, kernel, H)
    assert err <= tol, err


@pytest.mark.parametrize("mode", ["fp64", "fp32_fixup"])
def test_paper_full_cover_linear_field(ctx, mode):
    """Sec. 6.2: f = x over the 8-triangle [-1,1]^2 gives <f> = 0 and <grad f> = [1, 0]; a
    general linear field at an off-centre particle gives its value and gradient"""
    tris = full_cover_square(2).astype(np.float32)
    parts = np.array([[0.0, 0.0, 0.0, 0.0], [0.1, -0.05, 0.0, 0.0]], dtype=np.float32)
    v = tris.reshape(-1, 3, 2).astype(np.float64)
    vv = np.stack([v[..., 0], 1.0 + 2.0 * v[..., 0] - 3.0 * v[..., 1]], axis=-1).astype(np.float32)
    ctx.build_cells(_t(parts), _t(tris), 0.5)
    val, gr = ctx.field_integrals(_t(vv), "wendland_c4", mode)
    val, gr = val.double().cpu().numpy(), gr.double().cpu().numpy()
    tol = 1e-12 if mode == "fp64" else 2e-6
    x1, y1 = float(np.float32(0.1)), float(np.float32(-0.05))
    assert abs(val[0, 0]) < tol and np.allclose(gr[0, 0], [1.0, 0.0], atol=tol * 10)
    assert abs(val[1, 0] - x1) < tol and np.allclose(gr[1, 0], [1.0, 0.0], atol=tol * 10)
    assert abs(val[1, 1] - (1 + 2 * x1 - 3 * y1)) < tol * 10
    assert np.allclose(gr[1, 1], [2.0, -3.0], atol=tol * 50)


def test_constant_field_matches_boundary_integrals(ctx):
    w = W.wall_strip()
    parts, tris, H = w.particles, w.triangles, w.H
    vv = np.full((len(tris), 3, 1), 1.75, dtype=np.float32)
    g, gg, _ = ctx.boundary_integrals(_t(parts), _t(tris), "wendland_c2", H, -1, "fp64")
    val, gr = ctx.field_integrals(_t(vv), "wendland_c2", "fp64")
    g, gg = g.cpu().numpy(), gg.cpu().numpy()
    val, gr = val.cpu().numpy()[:, 0], gr.cpu().numpy()[:, 0]
    # the value uses the same gamma sums (to a few ulps: the two instantiations may contract
    # different multiply-adds); the gradient comes by parts, a different route
    assert np.max(np.abs(val - 1.75 * g)) <= 1e-14 * 1.75
    s = scales("wendland_c2", H, 0)[1]
    assert np.max(np.abs(gr - 1.75 * gg)) <= TOL_FP64 * 1.75 * s


def test_field_options_and_errors(ctx):
    import torch
    from paper_2507_21686_gb300._lib import Sph2dError
    w = W.wall_strip()
    parts, tris, H = w.particles, w.triangles, w.H
    vv = smooth_fields(tris, 4)
    ctx.build_cells(_t(parts), _t(tris), H)
    v4, g4 = ctx.field_integrals(_t(vv), "cubic_spline", "fp32_fixup")
    for nf in (1, 2, 3):
        v, g = ctx.field_integrals(_t(np.ascontiguousarray(vv[:, :, :nf])), "cubic_spline", "fp32_fixup")
        assert torch.equal(v, v4[:, :nf]) and torch.equal(g, g4[:, :nf])
    v0, g0 = ctx.field_integrals(_t(vv), "cubic_spline", "fp32_fixup", want_grad=False)
    # the same values from the kernel instantiation without the gradient, to a few ulps: the
    # two instantiations are compiled separately and may contract different multiply-adds
    assert g0 is None and float((v0 - v4).abs().max()) <= 1e-6 * float(v4.abs().max())
    v2, g2 = ctx.field_integrals(_t(vv), "cubic_spline", "fp32_fixup")
    assert torch.equal(v2, v4) and torch.equal(g2, g4)          # deterministic
    bad = np.zeros((len(tris), 3, 5), dtype=np.float32)
    with pytest.raises(Sph2dError, match="INVALID_ARG"):
        ctx.field_integrals(_t(bad), "wendland_c2", "fp64")
    with pytest.raises(Sph2dError, match="UNSUPPORTED"):
        ctx.field_integrals(_t(vv), "wendland_c2", "surrogate")
    from paper_2507_21686_gb300.api import Context
    c2 = Context(0)
    with pytest.raises(Sph2dError, match="NOT_BUILT"):
        c2.field_integrals(_t(vv), "wendland_c2", "fp64")
    c2.close()
