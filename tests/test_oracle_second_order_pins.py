"""Pins for the oracle's second-order adjoint quantities (d grad gamma / d nu_j): central
differences of the already-pinned divergence-theorem gradient with respect to each vertex and
to the particle, translation invariance, and symmetry of the particle Hessian."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2507_21686_gb300 import workloads as W

KERNELS = ["wendland_c2", "wendland_c4", "wendland_c6", "cubic_spline"]


def _cases(seed, n=12, H=0.7):
    rng = np.random.default_rng(seed)
    loc = W.surrogate_training_pairs(n, rng, lo=0.05, hi=1.5)
    xp = rng.uniform(-1, 1, size=(n, 2))
    tris = loc[:, 2:] * H + np.tile(xp, 3)
    # a triangle whose edge passes through the particle and one containing it
    tris = np.concatenate([tris, [[xp[0, 0] - 0.3 * H, xp[0, 1], xp[0, 0] + 0.4 * H, xp[0, 1], xp[0, 0], xp[0, 1] + 0.5 * H],
                                  [xp[1, 0] - 0.3 * H, xp[1, 1] - 0.2 * H, xp[1, 0] + 0.4 * H, xp[1, 1] - 0.1 * H,
                                   xp[1, 0], xp[1, 1] + 0.5 * H]]])
    xp = np.concatenate([xp, xp[:2]])
    return xp, tris, H


@pytest.mark.parametrize("kernel", KERNELS)
def test_vertex_jacobian_matches_central_differences(kernel):
    xp, tris, H = _cases(41)
    eps = 1e-6 * H
    for x, t in zip(xp, tris):
        J = oracle.grad_jacobian(kernel, H, x, t)
        fd = np.zeros((3, 2, 2))
        for j in range(3):
            for a in range(2):
                tp, tm = t.copy(), t.copy()
                tp[2 * j + a] += eps
                tm[2 * j + a] -= eps
                fd[j, :, a] = (oracle.pair(kernel, H, x, tp)[1:3] - oracle.pair(kernel, H, x, tm)[1:3]) / (2 * eps)
        scale = max(1.0 / H ** 2, np.max(np.abs(fd)))
        assert np.max(np.abs(J - fd)) < 1e-7 * scale


@pytest.mark.parametrize("kernel", KERNELS)
def test_particle_hessian_translation_and_symmetry(kernel):
    xp, tris, H = _cases(42)
    eps = 1e-6 * H
    for x, t in zip(xp, tris):
        J = oracle.grad_jacobian(kernel, H, x, t)
        Jx = -J.sum(axis=0)                    # moving the particle = moving every vertex back
        fd = np.zeros((2, 2))
        for a in range(2):
            xp_, xm_ = x.copy(), x.copy()
            xp_[a] += eps
            xm_[a] -= eps
            fd[:, a] = (oracle.pair(kernel, H, xp_, t)[1:3] - oracle.pair(kernel, H, xm_, t)[1:3]) / (2 * eps)
        scale = max(1.0 / H ** 2, np.max(np.abs(fd)))
        assert np.max(np.abs(Jx - fd)) < 1e-7 * scale
        assert abs(Jx[0, 1] - Jx[1, 0]) < 1e-9 * scale      # Hessian of gamma: symmetric
