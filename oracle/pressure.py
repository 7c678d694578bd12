"""Oracle for the boundary pressure coupling of Appendix A (TEST INFRASTRUCTURE ONLY; imported
by tests/ and the CPU legs of bench.py, never by the product path).  Plain numpy and the
pinned C oracle (kernel values, per-pair integrals, linear fields); no blocking or reordering.

Appendix A: the boundary's pressure acceleration of particle i is
    a_i = - int_Omega f(x') grad_x W(x_i - x') dx',   f = rho_0b (p(x')/rho_0b^2 + p_i/rho_i^2)
with the boundary density held at its rest value rho_0b, and the boundary pressure p(x') from
a moving-least-squares fit to the fluid particles' pressures (the appendix cites Band et al.'s
MLS extrapolation), in one of two models:
  model 1 (vertex pressure):  p at each triangle vertex by MLS, interpolated barycentrically;
      a_i = -(1/rho_0b) sum_T int_T p_T grad_x W  -  rho_0b p_i/rho_i^2 grad gamma_i
  model 2 (contact pressure): per pair one value p(x_iT) at the point of the triangle's
      boundary closest to x_i;
      a_i = - sum_T rho_0b (p(x_iT)/rho_0b^2 + p_i/rho_i^2) grad gamma_iT

MLS (the reading used here, since the appendix gives no formula): at a point b, minimise
    sum_j w_j (p_j - a - g . d_j)^2,  d_j = (x_j - b)/H,  w_j = V_j W(|x_j - b|)
over the fluid particles within H (V_j their volumes); p(b) = a.  Where the 3 x 3 normal
matrix is singular to 1e-6 relative (det <= 1e-6 (sum w)^3: fewer than three neighbours, or
all on a line) the zeroth-order (Shepard) average sum w p / sum w is used, and 0 where no
particle lies within H.
"""
from __future__ import annotations

import numpy as np

import oracle

MLS_SINGULAR = 1e-6


def mls_at(kernel, H, xs, vol, p, b):
    """MLS pressure at one point b from particles xs [N, 2], volumes vol [N], pressures p [N]
    (brute force over all particles)."""
    d = (np.asarray(xs, dtype=np.float64) - np.asarray(b, dtype=np.float64)) / H
    r = np.hypot(d[:, 0], d[:, 1])
    m = r < 1.0
    if not np.any(m):
        return 0.0
    C = oracle.kernel_C(kernel)
    vol = np.asarray(vol, dtype=np.float64)               # FP64 weights whatever the input type
    w = np.array([vol[j] * C / (H * H) * oracle.kernel_k(kernel, r[j]) for j in np.nonzero(m)[0]])
    dj = d[m]
    pj = np.asarray(p, dtype=np.float64)[m]
    X = np.stack([np.ones(len(dj)), dj[:, 0], dj[:, 1]], axis=1)
    A = X.T @ (w[:, None] * X)
    rhs = X.T @ (w * pj)
    sw = w.sum()
    if sw <= 0.0:
        return 0.0
    if np.linalg.det(A) <= MLS_SINGULAR * sw ** 3:
        return float((w * pj).sum() / sw)
    return float(np.linalg.solve(A, rhs)[0])


def mls_pressure(kernel, H, xs, vol, p, points):
    return np.array([mls_at(kernel, H, xs, vol, p, b) for b in np.asarray(points).reshape(-1, 2)])


def closest_on_boundary(x, tri):
    """point of the triangle's boundary (its three edges) closest to x"""
    v = np.asarray(tri, dtype=np.float64).reshape(3, 2)
    best, bd = None, np.inf
    for e in range(3):
        a, b = v[e], v[(e + 1) % 3]
        ab = b - a
        t = np.clip(np.dot(x - a, ab) / np.dot(ab, ab), 0.0, 1.0) if np.dot(ab, ab) > 0 else 0.0
        q = a + t * ab
        dd = np.hypot(*(x - q))
        if dd < bd:
            best, bd = q, dd
    return best


def boundary_pressure(kernel, H, particles, triangles, off, pair_tri, density, pressure, volume, rho0b,
                      model, sample=None):
    """a_i [len(sample), 2] for the particles in `sample` (indices; default all) of the culled
    pair list (off, pair_tri) of those particles; MLS over all particles."""
    parts = np.asarray(particles, dtype=np.float32)
    tris = np.asarray(triangles, dtype=np.float32).reshape(-1, 6)
    xs = parts[:, :2].astype(np.float64)
    idx = np.arange(len(parts)) if sample is None else np.asarray(sample)
    off = np.asarray(off, dtype=np.int64)
    pt = np.asarray(pair_tri, dtype=np.int64)
    pid = np.repeat(np.arange(len(idx)), np.diff(off))
    pairs = np.zeros((len(pt), 8))
    pairs[:, :2] = xs[idx][pid]
    pairs[:, 2:] = tris[pt]
    ref = oracle.pairs(kernel, H, pairs)                  # per-pair gamma, grad gamma, ...
    rho_i = np.asarray(density, dtype=np.float64)[idx]
    p_i = np.asarray(pressure, dtype=np.float64)[idx]
    acc = np.zeros((len(idx), 2))
    if model == 1:
        used = np.unique(pt)
        pv = np.zeros((len(tris), 3))
        for t in used:
            pv[t] = mls_pressure(kernel, H, xs, volume, pressure, tris[t].reshape(3, 2).astype(np.float64))
        fld = oracle.pairs_field(kernel, H, pairs, pv[pt])
        for q in range(len(pt)):
            i = pid[q]
            acc[i] -= fld[q, 1:3] / rho0b + rho0b * p_i[i] / rho_i[i] ** 2 * ref[q, 1:3]
    else:
        for q in range(len(pt)):
            i = pid[q]
            xc = closest_on_boundary(pairs[q, :2], tris[pt[q]])
            pc = mls_at(kernel, H, xs, volume, pressure, xc)
            acc[i] -= rho0b * (pc / rho0b ** 2 + p_i[i] / rho_i[i] ** 2) * ref[q, 1:3]
    return acc
