"""Adjoint kernel (sph2d_boundary_integrals_backward) vs the FP64 oracle: particle gradients
dL/dgamma * grad gamma, triangle-vertex gradients by the transport theorem, the translation
identity, central finite differences of the oracle, and the autograd Function."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300 import workloads as W
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


def oracle_backward(kernel, H, parts, tris, dg):
    off, pt = oracle.cull(parts, tris, H)
    g, gr, _, _ = oracle.particle_sums(kernel, H, parts, tris, off, pt, -1)
    pid = np.repeat(np.arange(len(parts)), np.diff(off))
    pairs = np.zeros((len(pt), 8))
    pairs[:, :2] = parts[pid, :2]
    pairs[:, 2:] = tris[pt]
    vg = oracle.pairs_vertex_grad(kernel, H, pairs) * dg[pid, None]
    dtri = np.zeros((len(tris), 6))
    np.add.at(dtri, pt, vg)
    return dg[:, None] * gr, dtri, g


@pytest.mark.parametrize("mode", ["fp64", "fp32_fixup"])
@pytest.mark.parametrize("kernel", ["wendland_c2", "wendland_c4", "cubic_spline"])
def test_backward_matches_oracle(ctx, kernel, mode):
    rng = np.random.default_rng(31)
    for w in (W.wall_strip(), W.box_obstacle(n=64)):
        dg = rng.normal(size=len(w.particles))
        ref_p, ref_t, _ = oracle_backward(kernel, w.H, w.particles, w.triangles, dg)
        dt = np.float64 if mode == "fp64" else np.float32
        dp, dtr = ctx.backward(_t(w.particles), _t(w.triangles), kernel, w.H, _t(dg.astype(dt)), mode)
        sg = scales(kernel, w.H, 0)[1] * np.abs(dg).max()
        tol = TOL_FP64 if mode == "fp64" else TOL_FP32
        assert rel_err(dp.cpu().numpy(), ref_p, sg).max() <= tol
        assert rel_err(dtr.cpu().numpy(), ref_t, sg).max() <= tol


def test_translation_identity(ctx):
    """sum over vertices of d gamma/d nu + d gamma/d x = 0 for every pair, hence globally."""
    w = W.box_obstacle(n=64)
    dg = np.random.default_rng(32).normal(size=len(w.particles))
    dp, dtr = ctx.backward(_t(w.particles), _t(w.triangles), "wendland_c4", w.H, _t(dg), "fp64")
    dp, dtr = dp.cpu().numpy(), dtr.cpu().numpy()
    tot = dp.sum(axis=0) + dtr.reshape(-1, 3, 2).sum(axis=(0, 1))
    mag = np.abs(dp).sum() + np.abs(dtr).sum()
    assert np.all(np.abs(tot) <= 1e-12 * mag)


def test_finite_differences_on_the_oracle(ctx):
    """Loss sum_i (gamma_i - gamma*_i)^2 with gamma* from a perturbed mesh: the adjoint's
    vertex gradients against central differences (step 1e-6 H) of the FP64 oracle."""
    w = W.adjoint_box(n=128, obstacle_cells=24)
    star = w.extra["target_triangles"]
    g, _, _ = ctx.boundary_integrals(_t(w.particles), _t(w.triangles), "wendland_c4", w.H, -1, "fp64")
    gs, _, _ = ctx.boundary_integrals(_t(w.particles), _t(star), "wendland_c4", w.H, -1, "fp64")
    dg = 2.0 * (g - gs)
    _, dtr = ctx.backward(_t(w.particles), _t(w.triangles), "wendland_c4", w.H, dg, "fp64")
    dtr, dg = dtr.cpu().numpy(), dg.cpu().numpy()
    off, pt = oracle.cull(w.particles, w.triangles, w.H)
    pid = np.repeat(np.arange(len(w.particles)), np.diff(off))
    rng = np.random.default_rng(33)
    busy = np.unique(pt[np.abs(dg[pid]) > 0])
    h = 1e-6 * w.H
    for t in rng.choice(busy, 12, replace=False):
        users = pid[pt == t]
        for j in rng.choice(6, 2, replace=False):
            fd = 0.0
            for i in users:
                tp = w.triangles[t].astype(np.float64).copy()
                tm = tp.copy()
                tp[j] += h
                tm[j] -= h
                xp = w.particles[i, :2].astype(np.float64)
                fd += dg[i] * (oracle.pair("wendland_c4", w.H, xp, tp)[0]
                               - oracle.pair("wendland_c4", w.H, xp, tm)[0]) / (2 * h)
            scale = scales("wendland_c4", w.H, 0)[1] * np.abs(dg).max()
            assert abs(dtr[t, j] - fd) <= 1e-7 * scale, (t, j, dtr[t, j], fd)


def test_autograd_function(ctx):
    import torch
    from paper_2507_21686_gb300.api import BoundaryGamma
    w = W.wall_strip()
    parts = _t(w.particles).double().requires_grad_(True)
    tris = _t(w.triangles).double().requires_grad_(True)
    target = torch.full((len(w.particles),), 0.2, dtype=torch.float64, device="cuda")
    g, _ = BoundaryGamma.apply(parts.float(), tris.float(), "wendland_c2", w.H, "fp64")
    loss = ((g - target) ** 2).sum()
    gp, gt = torch.autograd.grad(loss, [parts, tris])
    dp, dtr = ctx.backward(_t(w.particles), _t(w.triangles), "wendland_c2", w.H, (2 * (g - target)).detach(), "fp64")
    # the Function hands gradients back in the inputs' dtype (float32 here)
    assert torch.allclose(gp[:, :2], dp, rtol=1e-6, atol=1e-6 * dp.abs().max().item())
    assert torch.all(gp[:, 2:] == 0)
    assert torch.allclose(gt, dtr, rtol=1e-6, atol=1e-6 * dtr.abs().max().item())


def test_backward_rejects_bad_args(ctx):
    import torch
    from paper_2507_21686_gb300._lib import Sph2dError
    from paper_2507_21686_gb300.api import _ptr
    w = W.wall_strip()
    p, t = _t(w.particles), _t(w.triangles)
    dg = torch.zeros(len(w.particles), dtype=torch.float64, device="cuda")
    dp = torch.zeros((len(w.particles), 2), dtype=torch.float64, device="cuda")
    dt = torch.zeros((len(w.triangles), 6), dtype=torch.float64, device="cuda")
    st = ctx.lib.sph2d_boundary_integrals_backward(ctx.h, _ptr(p), p.shape[0], _ptr(t), t.shape[0], 0,
                                                   w.H, 2, _ptr(dg), None, _ptr(dp), _ptr(dt))
    assert st == 6                                       # surrogate mode: UNSUPPORTED
    with pytest.raises(Sph2dError):
        ctx.backward(p, t, "wendland_c2", -1.0, dg, "fp64")


# ---------------------------------------------------------------------------------------
# second order: dL/d grad gamma
# ---------------------------------------------------------------------------------------
def oracle_backward2(kernel, H, parts, tris, dg, dgr):
    """first-order part plus (d grad gamma / d x_i)^T G_i and (d grad gamma / d nu_j)^T G_i"""
    ref_p, ref_t, _ = oracle_backward(kernel, H, parts, tris, dg)
    off, pt = oracle.cull(parts, tris, H)
    pid = np.repeat(np.arange(len(parts)), np.diff(off))
    pairs = np.zeros((len(pt), 8))
    pairs[:, :2] = parts[pid, :2]
    pairs[:, 2:] = tris[pt]
    J = oracle.pairs_grad_jacobian(kernel, H, pairs)            # [P, 3, b, a]
    G = dgr[pid]                                                 # [P, 2]
    vt = np.einsum("pjba,pb->pja", J, G)                         # J_j^T G
    dtri = ref_t.copy()
    np.add.at(dtri, pt, vt.reshape(-1, 6))
    dp = ref_p.copy()
    np.add.at(dp, pid, -vt.sum(axis=1))
    return dp, dtri


@pytest.mark.parametrize("mode", ["fp64", "fp32_fixup"])
@pytest.mark.parametrize("kernel", ["wendland_c2", "wendland_c4", "wendland_c6", "cubic_spline"])
def test_second_order_backward_matches_oracle(ctx, kernel, mode):
    rng = np.random.default_rng(32)
    for w in (W.wall_strip(), W.box_obstacle(n=64)):
        n = len(w.particles)
        dg = rng.normal(size=n)
        dgr = rng.normal(size=(n, 2))
        ref_p, ref_t = oracle_backward2(kernel, w.H, w.particles, w.triangles, dg, dgr)
        dt = np.float64 if mode == "fp64" else np.float32
        dp, dtr = ctx.backward(_t(w.particles), _t(w.triangles), kernel, w.H, _t(dg.astype(dt)), mode,
                               d_grad=_t(dgr.astype(dt)))
        sg = scales(kernel, w.H, 0)[1]
        s = sg * (np.abs(dg).max() + np.abs(dgr).max() / w.H)     # grad-of-grad scales as 1/H^2
        tol = TOL_FP64 if mode == "fp64" else TOL_FP32
        assert rel_err(dp.cpu().numpy(), ref_p, s).max() <= tol
        assert rel_err(dtr.cpu().numpy(), ref_t, s).max() <= tol


def test_second_order_finite_differences(ctx):
    """L = sum_i G_i . grad gamma_i: the GPU's dL/dx and dL/dnu against central differences of
    the oracle's grad gamma (FP64)"""
    w = W.wall_strip()
    parts, tris, H = w.particles.astype(np.float64), w.triangles.astype(np.float64), w.H
    rng = np.random.default_rng(33)
    G = rng.normal(size=(len(parts), 2))
    dp, dtr = ctx.backward(_t(w.particles), _t(w.triangles), "cubic_spline", H,
                           _t(np.zeros(len(parts))), "fp64", d_grad=_t(G))
    dp, dtr = dp.cpu().numpy(), dtr.cpu().numpy()
    off, pt = oracle.cull(w.particles, w.triangles, H)

    def loss_particle(i, x):
        tot = 0.0
        for t in pt[off[i]:off[i + 1]]:
            tot += G[i] @ oracle.pair("cubic_spline", H, x, tris[t])[1:3]
        return tot

    eps = 1e-6 * H
    for i in np.flatnonzero(np.diff(off))[:6]:
        for a in range(2):
            xp_, xm_ = parts[i, :2].copy(), parts[i, :2].copy()
            xp_[a] += eps
            xm_[a] -= eps
            fd = (loss_particle(i, xp_) - loss_particle(i, xm_)) / (2 * eps)
            assert abs(dp[i, a] - fd) <= 1e-6 * max(1.0, abs(fd)) / H


# ---------------------------------------------------------------------------------------
# backward over the last build's pair list (no second cull)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["fp64", "fp32_fixup"])
@pytest.mark.parametrize("kernel", ["wendland_c2", "wendland_c4", "cubic_spline"])
def test_backward_from_pairs_is_the_full_backward(ctx, kernel, mode):
    """sph2d_backward_from_pairs after a forward call returns exactly what the rebuilding
    backward returns, with and without the grad gamma term"""
    import torch
    w = W.box_obstacle(n=64)
    rng = np.random.default_rng(41)
    dt = torch.float64 if mode == "fp64" else torch.float32
    dg = _t(rng.normal(size=len(w.particles))).to(dt)
    dgr = _t(rng.normal(size=(len(w.particles), 2))).to(dt)
    p, t = _t(w.particles), _t(w.triangles)
    for d_grad in (None, dgr):
        full_p, full_t = ctx.backward(p, t, kernel, w.H, dg, mode, d_grad)
        ctx.boundary_integrals(p, t, kernel, w.H, -1, mode)
        fp_p, fp_t = ctx.backward_from_pairs(kernel, dg, mode, d_grad)
        assert torch.equal(fp_p, full_p) and torch.equal(fp_t, full_t)


def test_backward_from_pairs_statuses(ctx):
    import torch
    from paper_2507_21686_gb300._lib import Sph2dError
    from paper_2507_21686_gb300.api import Context, _ptr
    fresh = Context(0)
    dg = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros((4, 6), dtype=torch.float64, device="cuda")
    assert fresh.lib.sph2d_backward_from_pairs(fresh.h, 0, 0, _ptr(dg), None, _ptr(out), _ptr(out)) == 4   # NOT_BUILT
    w = W.wall_strip()
    fresh.build_cells(_t(w.particles), _t(w.triangles), w.H)
    dg = torch.zeros(len(w.particles), dtype=torch.float64, device="cuda")
    with pytest.raises(Sph2dError, match="UNSUPPORTED"):
        fresh.backward_from_pairs("wendland_c2", dg, "surrogate")
    with pytest.raises(Sph2dError, match="INVALID_ARG"):
        fresh.backward_from_pairs(9, dg, "fp64")
    fresh.close()
