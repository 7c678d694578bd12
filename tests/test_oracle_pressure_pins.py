"""Pins for the oracle of Appendix A's boundary pressure coupling: MLS reproduces linear
pressure fields exactly and falls back to the neighbours' weighted average (by symmetry, their
mean) where the fit is singular; the closest boundary point by textbook cases; both pressure
models against the closed form for a constant pressure, -(p/rho_0b + rho_0b p/rho_i^2) grad
gamma_i; model 1 under a full cover against -grad p / rho_0b for a linear pressure."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import pressure as OP
from paper_2507_21686_gb300 import workloads as W
from paper_2507_21686_gb300.workloads import full_cover_square


def lattice(n, lo, hi, jitter, rng):
    g = np.linspace(lo, hi, n)
    x, y = np.meshgrid(g, g)
    pts = np.stack([x.ravel(), y.ravel()], axis=1)
    return pts + rng.uniform(-jitter, jitter, size=pts.shape)


@pytest.mark.parametrize("kernel", ["wendland_c2", "cubic_spline"])
def test_mls_reproduces_linear_pressure(kernel):
    rng = np.random.default_rng(51)
    xs = lattice(17, -1, 1, 0.02, rng)
    vol = rng.uniform(0.5, 1.5, size=len(xs))
    a, g = 2.0, np.array([0.7, -1.3])
    p = a + xs @ g
    pts = rng.uniform(-1.2, 1.2, size=(30, 2))             # inside and just outside the fluid
    got = OP.mls_pressure(kernel, 0.3, xs, vol, p, pts)
    assert np.allclose(got, a + pts @ g, atol=1e-11)


def test_mls_fallbacks():
    xs = np.array([[0.1, 0.0], [-0.1, 0.0], [5.0, 5.0]])
    vol = np.ones(3)
    p = np.array([3.0, 5.0, 100.0])
    # two neighbours on a line through the point, equal distance: their mean
    assert abs(OP.mls_at("wendland_c2", 0.5, xs, vol, p, (0.0, 0.0)) - 4.0) < 1e-14
    # one neighbour: its pressure; none: 0
    assert abs(OP.mls_at("wendland_c2", 0.5, xs, vol, p, (5.0, 5.2)) - 100.0) < 1e-14
    assert OP.mls_at("wendland_c2", 0.5, xs, vol, p, (-3.0, 2.0)) == 0.0


def test_closest_boundary_point():
    tri = np.array([0.0, 0.0, 1.0, 0.0, 0.0, 1.0])
    assert np.allclose(OP.closest_on_boundary(np.array([0.3, -0.5]), tri), [0.3, 0.0])
    assert np.allclose(OP.closest_on_boundary(np.array([-0.2, -0.3]), tri), [0.0, 0.0])
    assert np.allclose(OP.closest_on_boundary(np.array([1.0, 1.0]), tri), [0.5, 0.5])
    assert np.allclose(OP.closest_on_boundary(np.array([0.2, 0.1]), tri), [0.2, 0.0])   # inside


@pytest.mark.parametrize("model", [1, 2])
def test_constant_pressure_closed_form(model):
    """particles also fill the wall region, so that every vertex has MLS neighbours"""
    w = W.wall_strip()
    rng = np.random.default_rng(52)
    xs = lattice(33, -0.3, 1.0, 0.005, rng)
    parts = np.zeros((len(xs), 4), dtype=np.float32)
    parts[:, :2] = xs
    N = len(parts)
    rho = rng.uniform(900.0, 1100.0, size=N)
    pc, rho0b = 250.0, 1000.0
    p = np.full(N, pc)
    vol = np.full(N, (1.3 / 32) ** 2)
    sample = np.nonzero((xs[:, 1] > 0.0) & (xs[:, 1] < 0.15))[0][::3]
    off, pt = oracle.cull(parts[sample], w.triangles, w.H)
    acc = OP.boundary_pressure("wendland_c2", w.H, parts, w.triangles, off, pt, rho, p, vol, rho0b, model,
                               sample=sample)
    _, gg, _, _ = oracle.particle_sums("wendland_c2", w.H, parts[sample], w.triangles, off, pt, -1)
    ref = -(pc / rho0b + rho0b * pc / rho[sample, None] ** 2) * gg
    assert np.max(np.abs(acc - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(ref)) > 0.0


def test_model1_full_cover_linear_pressure():
    """support inside the [-1,1]^2 mesh: grad gamma = 0 and <grad p> = grad p, so a = -grad p /
    rho_0b whatever p_i is"""
    rng = np.random.default_rng(53)
    tris = full_cover_square(2).astype(np.float32)
    xs = lattice(17, -1, 1, 0.01, rng).astype(np.float32)
    parts = np.zeros((len(xs), 4), dtype=np.float32)
    parts[:, :2] = xs
    gp = np.array([30.0, -12.0])
    p = 100.0 + xs.astype(np.float64) @ gp
    rho = rng.uniform(900.0, 1100.0, size=len(xs))
    vol = np.full(len(xs), 0.125 ** 2)
    inner = np.nonzero(np.all(np.abs(xs) < 0.45, axis=1))[0][:12]
    H = 0.5
    off, pt = oracle.cull(parts[inner], tris, H)
    acc = OP.boundary_pressure("wendland_c4", H, parts, tris, off, pt, rho, p, vol, 1000.0, 1, sample=inner)
    assert np.allclose(acc, -gp / 1000.0, atol=1e-9)
