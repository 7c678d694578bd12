"""Parity at the full sizes the bench times, on sampled outputs the oracle computes one by one:
the adjoint on the 512^2 x 51,712 adjoint box (Wendland C4), boundary fields and the pressure
coupling on the 1024^2 x 197,120 box with obstacle.  Every expected value comes from the oracle
(its own cull of the sampled particles or triangles), none from the GPU path."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import pressure as OP
from paper_2507_21686_gb300 import workloads as W
from paper_2507_21686_gb300.workloads import field_node_positions, hydrostatic_state
from tests.helpers import TOL_FP32, rel_err, scales

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


@pytest.fixture(scope="module")
def box():
    return W.box_obstacle()


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def near_sample(w, rng, n_near, n_any):
    """particles that see triangles (found by the oracle's cull of a random superset) and a few
    random ones"""
    cand = rng.choice(len(w.particles), 20 * n_near, replace=False)
    off, _ = oracle.cull(w.particles[cand], w.triangles, w.H)
    near = cand[np.diff(off) > 0]
    pick = np.concatenate([near[:n_near], rng.choice(len(w.particles), n_any, replace=False)])
    return np.unique(pick)


def test_adjoint_box_full_size_sampled(ctx):
    """backward of L = sum (gamma - gamma*)^2 style weights on the bench's adjoint workload:
    particle gradients on sampled particles, vertex gradients on sampled triangles"""
    w = W.adjoint_box()
    rng = np.random.default_rng(81)
    dg = rng.normal(size=len(w.particles)).astype(np.float32)
    dp, dtr = ctx.backward(_t(w.particles), _t(w.triangles), "wendland_c4", w.H, _t(dg), "fp32_fixup")
    dp, dtr = dp.double().cpu().numpy(), dtr.double().cpu().numpy()
    sg = scales("wendland_c4", w.H, 0)[1] * np.abs(dg).max()
    # particles
    ps = near_sample(w, rng, 60, 20)
    off, pt = oracle.cull(w.particles[ps], w.triangles, w.H)
    _, ogr, _, _ = oracle.particle_sums("wendland_c4", w.H, w.particles[ps], w.triangles, off, pt, -1)
    assert rel_err(dp[ps], dg[ps, None].astype(np.float64) * ogr, sg).max() <= TOL_FP32
    # triangles: all pairs of the sampled triangles, from the oracle's cull of every particle
    ts = np.unique(np.concatenate([rng.choice(len(w.triangles), 40, replace=False),
                                   np.arange(0, len(w.triangles), len(w.triangles) // 10)]))
    off2, pt2 = oracle.cull(w.particles, w.triangles[ts], w.H)
    pid = np.repeat(np.arange(len(w.particles)), np.diff(off2))
    pairs = np.zeros((len(pt2), 8))
    pairs[:, :2] = w.particles[pid, :2]
    pairs[:, 2:] = w.triangles[ts][pt2]
    vg = oracle.pairs_vertex_grad("wendland_c4", w.H, pairs) * dg[pid, None].astype(np.float64)
    ref = np.zeros((len(ts), 6))
    np.add.at(ref, pt2, vg)
    assert rel_err(dtr[ts], ref, sg).max() <= TOL_FP32
    assert np.abs(ref).max() > 0


@pytest.mark.parametrize("order,mode", [(1, "fp32_fixup"), (3, "fp32_hybrid")])
def test_fields_full_size_sampled(ctx, box, order, mode):
    """the bench's fields (rho = 1 + xy/4 and rho u at the element nodes), Wendland C4"""
    w = box
    v = field_node_positions(w.triangles, order)
    rho = 1.0 + 0.25 * v[..., 0] * v[..., 1]
    u = np.sin(3 * v[..., 0]) + np.cos(2 * v[..., 1])
    vv = np.stack([rho, rho * u], axis=-1).astype(np.float32)
    ctx.build_cells(_t(w.particles), _t(w.triangles), w.H)
    val, gr = ctx.field_integrals(_t(vv), "wendland_c4", mode, order=order)
    val, gr = val.double().cpu().numpy(), gr.double().cpu().numpy()
    rng = np.random.default_rng(82 + order)
    ps = near_sample(w, rng, 80, 20)
    off, pt = oracle.cull(w.particles[ps], w.triangles, w.H)
    rv, rg = oracle.particle_field_sums_p("wendland_c4", w.H, w.particles[ps], w.triangles, off, pt, order, vv)
    A = np.max(np.abs(vv), axis=(0, 1))
    sc = scales("wendland_c4", w.H, 0)
    ev = np.abs(val[ps] - rv) / np.maximum(np.abs(rv), A[None, :] * sc[0])
    eg = np.abs(gr[ps] - rg) / np.maximum(np.abs(rg), A[None, :, None] * sc[1])
    assert max(ev.max(), eg.max()) <= TOL_FP32


@pytest.mark.parametrize("model", [1, 2])
def test_pressure_full_size_sampled(ctx, box, model):
    """the bench's pressure leg: hydrostatic state, Wendland C4, FP32 + fix-up"""
    w = box
    st = hydrostatic_state(w.particles, 1.0 / 1024, 2)
    ctx.build_cells(_t(w.particles), _t(w.triangles), w.H)
    acc = ctx.boundary_pressure(_t(st["density"]), _t(st["pressure"]), _t(st["volume"]), st["rho0_b"],
                                "wendland_c4", "fp32_fixup", model).double().cpu().numpy()
    rng = np.random.default_rng(84 + model)
    ps = near_sample(w, rng, 24, 0)
    off, pt = oracle.cull(w.particles[ps], w.triangles, w.H)
    # The MLS points of a sampled particle (its triangles' vertices, at most H + the longest edge
    # away, and its contact points, within H) have their neighbours within another H: the
    # particles within 3 H of the sample hold every neighbourhood, so the oracle's brute force
    # runs over those only.
    xy = w.particles[:, :2].astype(np.float64)
    keep = np.zeros(len(xy), dtype=bool)
    for i in ps:
        keep |= np.hypot(xy[:, 0] - xy[i, 0], xy[:, 1] - xy[i, 1]) < 3.0 * w.H
    sub = np.nonzero(keep)[0]
    remap = np.full(len(xy), -1)
    remap[sub] = np.arange(len(sub))
    ref = OP.boundary_pressure("wendland_c4", w.H, w.particles[sub], w.triangles, off, pt, st["density"][sub],
                               st["pressure"][sub], st["volume"][sub], st["rho0_b"], model, sample=remap[ps])
    pmax = float(st["pressure"].max())
    sc = (pmax / st["rho0_b"] + st["rho0_b"] * pmax / float(st["density"].min()) ** 2) * scales("wendland_c4", w.H, 0)[1]
    assert np.max(np.abs(acc[ps] - ref)) / sc <= TOL_FP32
    assert np.abs(ref).max() > 1e-3 * sc
