"""The allocation-free entry point (sph2d_pair_list_integrals_noalloc) against the regular
per-particle integrals and, on the wall strip, against the FP64 oracle element by element,
called through the C-ABI.

Callers that cannot allocate device memory while they run (pools that forbid cudaMalloc in a
solver step, frameworks owning all device memory) use this entry point with their own
buffers; its scratch is a fixed device array inside the library.  This file is collected last
so that a failure here comes after every other test has run."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300 import workloads as W
from tests.helpers import TOL_FP32, TOL_FP64, rel_err, scales

pytestmark = pytest.mark.gpu

KNAMES = ["wendland_c2", "wendland_c4", "wendland_c6", "cubic_spline"]


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


def _call(lib, parts, tris, off, tri, kernel, H, mode, gamma, grad):
    import torch
    from paper_2507_21686_gb300.api import _ptr
    st = torch.cuda.current_stream().cuda_stream
    return lib.sph2d_pair_list_integrals_noalloc(
        _ptr(parts), parts.shape[0], _ptr(tris), tris.shape[0], _ptr(off), _ptr(tri), tri.numel(),
        kernel, float(H), mode, _ptr(gamma), _ptr(grad), ctypes.c_void_p(st))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kernel", [0, 3])
def test_noalloc_matches_regular_entry_point(ctx, kernel, mode):
    import torch
    dt = torch.float64 if mode == 0 else torch.float32
    tol = TOL_FP64 if mode == 0 else TOL_FP32
    for w in (W.wall_strip(), W.box_obstacle(n=128)):
        parts = torch.from_numpy(w.particles).cuda()
        tris = torch.from_numpy(w.triangles).cuda()
        g_ref, gr_ref, _ = ctx.boundary_integrals(parts, tris, kernel, w.H, -1, "fp64" if mode == 0 else "fp32_fixup")
        off, tri = ctx.pair_list()
        ref = torch.cat([g_ref[:, None], gr_ref], 1).double().cpu().numpy()
        orc = None
        if w.name.startswith("wall_strip"):
            o_off, o_pt = oracle.cull(w.particles, w.triangles, w.H)
            assert np.array_equal(off.cpu().numpy(), o_off) and np.array_equal(tri.cpu().numpy(), o_pt)
            og, ogr, _, _ = oracle.particle_sums(KNAMES[kernel], w.H, w.particles, w.triangles, o_off, o_pt, -1)
            orc = np.concatenate([og[:, None], ogr], axis=1)
        for _ in range(2):                              # two calls in a row share the scratch
            g = torch.full((parts.shape[0],), float("nan"), dtype=dt, device="cuda")
            gr = torch.full((parts.shape[0], 2), float("nan"), dtype=dt, device="cuda")
            assert _call(ctx.lib, parts, tris, off, tri, kernel, w.H, mode, g, gr) == 0
            got = torch.cat([g[:, None], gr], 1).double().cpu().numpy()
            assert rel_err(got, ref, scales(kernel, w.H, 0)).max() <= tol
            if orc is not None:
                assert rel_err(got, orc, scales(kernel, w.H, 0)).max() <= tol


def test_noalloc_rejects_lists_beyond_its_scratch(ctx):
    import torch
    w = W.wall_strip()
    parts = torch.from_numpy(w.particles).cuda()
    tris = torch.from_numpy(w.triangles).cuda()
    ctx.build_cells(parts, tris, w.H)
    off, tri = ctx.pair_list()
    g = torch.zeros(parts.shape[0], dtype=torch.float64, device="cuda")
    from paper_2507_21686_gb300.api import _ptr
    too_many = 32 * ((8 << 20) - 256) // 48 + 32      # above the FP64 limit
    st = ctx.lib.sph2d_pair_list_integrals_noalloc(
        _ptr(parts), parts.shape[0], _ptr(tris), tris.shape[0], _ptr(off), _ptr(tri), too_many,
        0, float(w.H), 0, _ptr(g), None, None)
    assert st == 3                                      # SPH2D_ERR_CAPACITY, nothing enqueued
