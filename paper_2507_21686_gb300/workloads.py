"""Seeded synthetic inputs for the 2-D SPH boundary-integral workloads.

This module is the ONLY code shared by the FP64 oracle (``oracle/``) and the CUDA path.
It holds none of the method's arithmetic: jittered particle lattices, structured
triangulated wall meshes, and random (particle, triangle) pair geometry, all drawn from
``numpy.random.default_rng(seed)`` so that both sides see bit-identical inputs.

Layouts (what the C-ABI consumes):
  particles  float32 [N, 4]  (x, y, 0, 0)        -- float4 per particle
  triangles  float32 [M, 6]  (x0, y0, x1, y1, x2, y2)
  pairs      float64 [P, 8]  (px, py, x0, y0, x1, y1, x2, y2)  -- per-pair entry point

The workloads model the paper's setting (Sec. 2, Eq. boundaryint: fluid particles next to
a boundary built from disjoint triangles; Sec. 6.2: [-1,1]^2 meshes) at the sizes listed
in ``WORKLOADS``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KERNEL_IDS = {"wendland_c2": 0, "wendland_c4": 1, "wendland_c6": 2, "cubic_spline": 3}


# ----------------------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------------------
def jittered_lattice(n: int, dx: float, jitter: float, rng: np.random.Generator,
                     origin=(0.0, 0.0)) -> np.ndarray:
    """n*n particles at (origin + (i+1/2, j+1/2) dx), each axis jittered by U(-jitter, jitter)*dx.

    Index = j*n + i.  Returns float32 [n*n, 4] with columns (x, y, 0, 0).
    """
    i = np.arange(n, dtype=np.float64)
    xs, ys = np.meshgrid(i, i, indexing="xy")        # ys varies along rows (j), xs along i
    x = origin[0] + (xs.ravel() + 0.5) * dx
    y = origin[1] + (ys.ravel() + 0.5) * dx
    j = rng.uniform(-jitter, jitter, size=(n * n, 2)) * dx
    out = np.zeros((n * n, 4), dtype=np.float32)
    out[:, 0] = (x + j[:, 0]).astype(np.float32)
    out[:, 1] = (y + j[:, 1]).astype(np.float32)
    return out


def structured_mesh(origin, cell, nx: int, ny: int, cell_mask: np.ndarray,
                    rng: np.random.Generator, jitter_frac: float = 0.1,
                    cell_y: float | None = None) -> np.ndarray:
    """Triangulate the cells of an (nx x ny) grid selected by ``cell_mask[j, i]``.

    Vertex (i, j) sits at origin + (i*cell, j*cell_y).  A vertex whose four surrounding
    cells are all in the mesh is an interior vertex and is jittered by
    U(-jitter_frac, jitter_frac) of a cell per axis; surface vertices stay fixed, so walls
    remain straight.  Each cell (v00, v10, v11, v01) is split on its (0,0)-(1,1) diagonal
    into (v00, v10, v11) and (v00, v11, v01), both counter-clockwise.  Cells are emitted in
    row-major order (j outer).  Returns float32 [M, 6].
    """
    cy = cell if cell_y is None else cell_y
    mask = np.asarray(cell_mask, dtype=bool)
    assert mask.shape == (ny, nx)
    vi, vj = np.meshgrid(np.arange(nx + 1, dtype=np.float64),
                         np.arange(ny + 1, dtype=np.float64), indexing="xy")
    vx = origin[0] + vi * cell
    vy = origin[1] + vj * cy
    # interior vertex: all four adjacent cells present (outer grid boundary is never interior)
    pad = np.zeros((ny + 2, nx + 2), dtype=bool)
    pad[1:-1, 1:-1] = mask
    interior = pad[:-1, :-1] & pad[:-1, 1:] & pad[1:, :-1] & pad[1:, 1:]
    jit = rng.uniform(-jitter_frac, jitter_frac, size=(ny + 1, nx + 1, 2))
    vx = np.where(interior, vx + jit[..., 0] * cell, vx)
    vy = np.where(interior, vy + jit[..., 1] * cy, vy)
    cj, ci = np.nonzero(mask)                       # row-major order
    x00, y00 = vx[cj, ci], vy[cj, ci]
    x10, y10 = vx[cj, ci + 1], vy[cj, ci + 1]
    x11, y11 = vx[cj + 1, ci + 1], vy[cj + 1, ci + 1]
    x01, y01 = vx[cj + 1, ci], vy[cj + 1, ci]
    m = len(cj)
    tris = np.empty((2 * m, 6), dtype=np.float64)
    tris[0::2] = np.stack([x00, y00, x10, y10, x11, y11], axis=1)
    tris[1::2] = np.stack([x00, y00, x11, y11, x01, y01], axis=1)
    return tris.astype(np.float32)


def box_band_mesh(n: int, dx: float, band: int, rng: np.random.Generator) -> np.ndarray:
    """Closed box wall: the band [-band*dx, 1+band*dx]^2 minus [0,1]^2, cells of size dx."""
    tot = n + 2 * band
    mask = np.ones((tot, tot), dtype=bool)
    mask[band:band + n, band:band + n] = False
    return structured_mesh((-band * dx, -band * dx), dx, tot, tot, mask, rng)


def solid_square_mesh(lo: float, cells: int, dx: float, rng: np.random.Generator) -> np.ndarray:
    """Solid square obstacle [lo, lo+cells*dx]^2 meshed at cell size dx."""
    mask = np.ones((cells, cells), dtype=bool)
    return structured_mesh((lo, lo), dx, cells, cells, mask, rng)


# ----------------------------------------------------------------------------------------
# per-pair stress geometry (local frame, H = 1, particle at the origin)
# ----------------------------------------------------------------------------------------
def _point_triangle_distance(px, py, t):
    """Euclidean distance from points to closed triangles (placement only, float64)."""
    best = np.full(px.shape, np.inf)
    inside_pos = np.ones(px.shape, dtype=bool)
    inside_neg = np.ones(px.shape, dtype=bool)
    for a, b in ((0, 1), (1, 2), (2, 0)):
        ax, ay, bx, by = t[:, 2 * a], t[:, 2 * a + 1], t[:, 2 * b], t[:, 2 * b + 1]
        ex, ey = bx - ax, by - ay
        wx, wy = px - ax, py - ay
        l2 = ex * ex + ey * ey
        s = np.clip(np.where(l2 > 0, (wx * ex + wy * ey) / np.where(l2 > 0, l2, 1), 0), 0, 1)
        dxq, dyq = wx - s * ex, wy - s * ey
        best = np.minimum(best, np.hypot(dxq, dyq))
        cr = ex * wy - ey * wx
        inside_pos &= cr >= 0
        inside_neg &= cr <= 0
    return np.where(inside_pos | inside_neg, 0.0, best)


def _random_shape(rng, count, kind):
    """Triangles (float64 [count, 6]) centred near 0 with longest edge 1 before scaling."""
    out = np.empty((count, 6))
    filled = 0
    while filled < count:
        k = (count - filled) * 2 + 16
        if kind == "generic":
            ang = rng.uniform(0, 2 * np.pi, size=(k, 3))
            pts = np.stack([np.cos(ang), np.sin(ang)], axis=2)       # on the unit circle
            e = [pts[:, 1] - pts[:, 0], pts[:, 2] - pts[:, 1], pts[:, 0] - pts[:, 2]]
            ln = np.stack([np.hypot(v[:, 0], v[:, 1]) for v in e], axis=1)
            # interior angles by the law of cosines; keep triangles with all angles >= 15 deg
            a, b, c = ln[:, 1], ln[:, 2], ln[:, 0]
            with np.errstate(invalid="ignore", divide="ignore"):
                A0 = np.arccos(np.clip((b * b + c * c - a * a) / (2 * b * c), -1, 1))
                A1 = np.arccos(np.clip((a * a + c * c - b * b) / (2 * a * c), -1, 1))
            A2 = np.pi - A0 - A1
            ok = (np.minimum(np.minimum(A0, A1), A2) >= np.deg2rad(15.0)) & np.isfinite(A0)
            pts = pts[ok] / ln[ok].max(axis=1)[:, None, None]
            tri = pts.reshape(-1, 6)
        else:  # sliver: base of length 1, apex at height 1/A above a point in [-0.5, 1.5]
            A = np.exp(rng.uniform(math.log(10.0), math.log(1e6), size=k))
            u = rng.uniform(-0.5, 1.5, size=k)
            tri = np.stack([np.zeros(k), np.zeros(k), np.ones(k), np.zeros(k), u, 1.0 / A], axis=1)
            tri -= np.tile([0.5, 0.0], 3)
            th = rng.uniform(0, 2 * np.pi, size=k)
            c, s = np.cos(th), np.sin(th)
            x, y = tri[:, 0::2].copy(), tri[:, 1::2].copy()
            tri[:, 0::2], tri[:, 1::2] = c[:, None] * x - s[:, None] * y, s[:, None] * x + c[:, None] * y
        take = min(len(tri), count - filled)
        out[filled:filled + take] = tri[:take]
        filled += take
    return out


def _place_within_support(rng, shapes):
    """Translate each shape by a random offset, uniform over the region where its
    distance to the origin is < 1 (rejection sampling)."""
    n = len(shapes)
    out = np.empty_like(shapes)
    todo = np.arange(n)
    while len(todo):
        t = shapes[todo]
        cx, cy = t[:, 0::2].mean(axis=1), t[:, 1::2].mean(axis=1)
        rad = np.max(np.hypot(t[:, 0::2] - cx[:, None], t[:, 1::2] - cy[:, None]), axis=1) + 1.0
        ox = rng.uniform(-1, 1, size=len(todo)) * rad - cx
        oy = rng.uniform(-1, 1, size=len(todo)) * rad - cy
        moved = t + np.tile(np.stack([ox, oy], axis=1), 3)
        d = _point_triangle_distance(np.zeros(len(todo)), np.zeros(len(todo)), moved)
        ok = d < 1.0
        out[todo[ok]] = moved[ok]
        todo = todo[~ok]
    return out


def surrogate_training_pairs(count: int, rng: np.random.Generator, lo: float = 0.08,
                             hi: float = 0.5) -> np.ndarray:
    """Training and test pairs for the learned surrogate (local frame, H = 1): generic
    triangles (all angles >= 15 deg) with longest edge logU[lo, hi], placed uniformly over
    the region where they overlap the support.  float64 [count, 8] (particle at 0)."""
    size = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    shapes = _random_shape(rng, count, "generic") * size[:, None]
    pairs = np.zeros((count, 8))
    pairs[:, 2:] = _place_within_support(rng, shapes)
    return pairs


def stress_pairs(count: int, rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """Precision-stress pairs in the local frame (H = 1, particle at the origin).

    Three equal classes (label 0/1/2): generic triangles (all angles >= 15 deg); slivers
    with aspect ratio A ~ logU[10, 1e6]; near-singular pairs with the particle at
    delta ~ logU[1e-16, 1e-8] from an edge line (half) or a vertex (half), delta = 0 exactly
    for 1/64 of them.  Triangle size (longest edge) s ~ logU[1e-3, 10].
    Returns (pairs float64 [count, 8], labels int8 [count]).
    """
    n0 = count // 3
    n1 = count // 3
    n2 = count - n0 - n1
    size = np.exp(rng.uniform(math.log(1e-3), math.log(10.0), size=count))
    gen = _random_shape(rng, n0, "generic") * size[:n0, None]
    sl = _random_shape(rng, n1, "sliver") * size[n0:n0 + n1, None]
    gen = _place_within_support(rng, gen)
    sl = _place_within_support(rng, sl)
    # near-singular: generic shapes, particle pinned near an edge line or a vertex
    ns = _random_shape(rng, n2, "generic") * size[n0 + n1:, None]
    delta = np.exp(rng.uniform(math.log(1e-16), math.log(1e-8), size=n2))
    zero = rng.uniform(size=n2) < 1.0 / 64.0
    delta[zero] = 0.0
    on_edge = rng.uniform(size=n2) < 0.5
    which = rng.integers(0, 3, size=n2)
    lam = rng.uniform(0.0, 1.0, size=n2)
    lam[zero & on_edge] = 0.5              # exact midpoint keeps the zero-distance case exact
    side = np.where(rng.uniform(size=n2) < 0.5, -1.0, 1.0)
    phi = rng.uniform(0, 2 * np.pi, size=n2)
    rel = np.empty_like(ns)
    for r in range(n2):
        t = ns[r].reshape(3, 2)
        a = t[which[r]]
        b = t[(which[r] + 1) % 3]
        if on_edge[r]:
            e = b - a
            q_minus_a = lam[r] * e                                     # particle foot on the edge
            nrm = np.array([-e[1], e[0]]) / math.hypot(e[0], e[1])
            off = side[r] * delta[r] * nrm
            rel[r] = (t - a - q_minus_a - off).ravel() if not zero[r] else (t - a - q_minus_a).ravel()
            if zero[r]:
                # a, b relative to the midpoint are exactly -e/2 and +e/2
                rel[r, 2 * which[r]:2 * which[r] + 2] = -0.5 * e
                bi = (which[r] + 1) % 3
                rel[r, 2 * bi:2 * bi + 2] = 0.5 * e
        else:
            off = delta[r] * np.array([math.cos(phi[r]), math.sin(phi[r])])
            rel[r] = (t - a - off).ravel()
            if zero[r]:
                rel[r, 2 * which[r]:2 * which[r] + 2] = 0.0
    pairs = np.zeros((count, 8))
    pairs[:n0, 2:] = gen
    pairs[n0:n0 + n1, 2:] = sl
    pairs[n0 + n1:, 2:] = rel
    labels = np.concatenate([np.zeros(n0), np.ones(n1), np.full(n2, 2)]).astype(np.int8)
    return pairs, labels


def surrogate_pairs(count: int, rng: np.random.Generator) -> np.ndarray:
    """Training pairs for the learned surrogate: triangle size logU[1e-3, 10], distance of
    the triangle to the particle logU[1e-4, 1], random pose (local frame, H = 1)."""
    size = np.exp(rng.uniform(math.log(1e-3), math.log(10.0), size=count))
    shapes = _random_shape(rng, count, "generic") * size[:, None]
    dist = np.exp(rng.uniform(math.log(1e-4), 0.0, size=count))
    # place the closest vertex at the requested distance in a random direction, then push
    # the triangle outward so that the vertex is the nearest point (a valid, seeded pose)
    phi = rng.uniform(0, 2 * np.pi, size=count)
    d = np.stack([np.cos(phi), np.sin(phi)], axis=1)
    v = shapes.reshape(count, 3, 2)
    proj = np.einsum("nkj,nj->nk", v, d)
    k = np.argmin(proj, axis=1)
    anchor = v[np.arange(count), k]
    v = v - anchor[:, None, :] + (dist[:, None] * d)[:, None, :]
    pairs = np.zeros((count, 8))
    pairs[:, 2:] = v.reshape(count, 6)
    return pairs


# ----------------------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    H: float
    kernels: list
    moment_degree: int
    particles: np.ndarray | None = None          # float32 [N, 4]
    triangles: np.ndarray | None = None          # float32 [M, 6]
    pairs: np.ndarray | None = None              # float64 [P, 8] (per-pair workloads)
    labels: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def wall_strip(seed: int = 1) -> Workload:
    """1,024 particles (32x32 jittered lattice, dx=1/32, +-0.25dx) over a 64-triangle wall
    (8x4 cells over [0,1]x[-0.25,0], interior vertices jittered +-0.1 cell); H = 4dx,
    Wendland C2, gamma and grad gamma."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / 32.0
    parts = jittered_lattice(32, dx, 0.25, rng)
    mask = np.ones((4, 8), dtype=bool)
    tris = structured_mesh((0.0, -0.25), 0.125, 8, 4, mask, rng, cell_y=0.0625)
    return Workload("wall_strip_1k_x_64", 4 * dx, ["wendland_c2"], -1, parts, tris)


def box_obstacle(seed: int = 2, n: int = 1024, obstacle_cells: int | None = None) -> Workload:
    """n^2 jittered particles in the unit square, H = 4dx, inside a closed box band
    (8 cells thick) with a solid square obstacle [0.375, 0.625]^2, all meshed at dx.
    n = 1024 gives 1,048,576 particles and 197,120 triangles."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    parts = jittered_lattice(n, dx, 0.25, rng)
    band = box_band_mesh(n, dx, 8, rng)
    oc = obstacle_cells if obstacle_cells is not None else n // 4
    lo = 0.5 - 0.5 * oc * dx
    obs = solid_square_mesh(lo, oc, dx, rng)
    tris = np.concatenate([band, obs], axis=0)
    return Workload(f"box_obstacle_{n * n}_x_{len(tris)}", 4 * dx,
                    ["wendland_c2", "wendland_c4", "cubic_spline"], 3, parts, tris)


def hydrostatic_state(particles: np.ndarray, dx: float, seed: int) -> dict:
    """Fluid state for the boundary pressure coupling: rest density 1000 with +-1% noise,
    hydrostatic pressure 1000 g (1 - y) (g = 9.81) with +-2% noise, volumes dx^2; boundary rest
    density rho_0b = 1000.  float32 arrays density, pressure, volume and rho0_b."""
    rng = np.random.default_rng(seed + 100)
    N = len(particles)
    y = np.asarray(particles)[:, 1].astype(np.float64)
    dens = 1000.0 * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, size=N))
    pres = 1000.0 * 9.81 * (1.0 - y) * (1.0 + 0.02 * rng.uniform(-1.0, 1.0, size=N))
    return {"density": dens.astype(np.float32), "pressure": pres.astype(np.float32),
            "volume": np.full(N, dx * dx, dtype=np.float32), "rho0_b": 1000.0}


def hydrostatic_box(seed: int = 6, n: int = 1024, obstacle_cells: int | None = None) -> Workload:
    """The box-with-obstacle geometry of box_obstacle(seed, n) with the fluid state of
    hydrostatic_state in extra."""
    w = box_obstacle(seed, n, obstacle_cells)
    w.extra = hydrostatic_state(w.particles, 1.0 / n, seed)
    w.name = f"hydrostatic_box_{len(w.particles)}_x_{len(w.triangles)}"
    return w


def precision_stress(seed: int = 3, count: int = 262_144) -> Workload:
    """262,144 local-frame pairs (generic / sliver / near-singular), Wendland C2, C4, C6."""
    rng = np.random.default_rng(seed)
    pairs, labels = stress_pairs(count, rng)
    return Workload(f"precision_stress_{count}", 1.0,
                    ["wendland_c2", "wendland_c4", "wendland_c6"], 3, pairs=pairs, labels=labels)


def adjoint_box(seed: int = 4, n: int = 512, obstacle_cells: int = 96,
                target_seed: int = 104) -> Workload:
    """512^2 particles, box band at dx plus a 96x96-cell solid obstacle (51,712 triangles),
    Wendland C4; the target gamma* comes from the same mesh with every vertex perturbed
    by U(+-0.05 cell) (seed 104)."""
    w = box_obstacle(seed, n, obstacle_cells)
    trng = np.random.default_rng(target_seed)
    pert = w.triangles.astype(np.float64) + trng.uniform(-0.05, 0.05, size=w.triangles.shape) / n
    w.name = f"adjoint_box_{n * n}_x_{len(w.triangles)}"
    w.kernels = ["wendland_c4"]
    w.moment_degree = -1
    w.extra["target_triangles"] = pert.astype(np.float32)
    return w


def surrogate_box(seed: int = 5, n: int = 2048, obstacle_cells: int = 660) -> Workload:
    """2048^2 particles, box band plus a 660x660-cell obstacle (1,002,784 triangles), C2."""
    w = box_obstacle(seed, n, obstacle_cells)
    w.name = f"surrogate_box_{n * n}_x_{len(w.triangles)}"
    w.kernels = ["wendland_c2"]
    w.moment_degree = -1
    return w


# node lattice of the order-k Lagrange triangle (barycentric indices / k), in the node order of
# sph2d_field_integrals_p: vertices, the nodes inside edges (0,1), (1,2), (2,0) from the
# first vertex to the second, then the interior node
_NODE_LATTICE = {
    1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
    2: [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (0, 1, 1), (1, 0, 1)],
    3: [(3, 0, 0), (0, 3, 0), (0, 0, 3), (2, 1, 0), (1, 2, 0), (0, 2, 1), (0, 1, 2), (1, 0, 2), (2, 0, 1),
        (1, 1, 1)],
}


def field_node_positions(triangles: np.ndarray, order: int) -> np.ndarray:
    """World positions [M, nodes, 2] of the order-k field nodes of each triangle (float64), for
    sampling a field function into node values."""
    t = np.asarray(triangles, dtype=np.float64).reshape(-1, 3, 2)
    w = np.asarray(_NODE_LATTICE[order], dtype=np.float64) / order
    return np.einsum("nj,mjc->mnc", w, t)


def full_cover_square(n_side: int = 2) -> np.ndarray:
    """Triangulation of [-1,1]^2 into 2*n_side^2 triangles (n_side=2: the paper's 8-triangle
    mesh of Sec. 6.2; n_side=... finer meshes for additivity checks).  float64 [M, 6]."""
    g = np.linspace(-1.0, 1.0, n_side + 1)
    tris = []
    for j in range(n_side):
        for i in range(n_side):
            x0, x1, y0, y1 = g[i], g[i + 1], g[j], g[j + 1]
            tris.append([x0, y0, x1, y0, x1, y1])
            tris.append([x0, y0, x1, y1, x0, y1])
    return np.asarray(tris, dtype=np.float64)
