"""Pins for the FP64 oracle: each check compares the oracle with something other than itself
(closed forms in exact rational arithmetic, 1-D library quadrature, brute-force 2-D
quadrature, invariants of the definition, exact rational culling), chosen so that a dropped
term, a wrong sign, a transposed operand or a wrong constant fails at least one of them.
``test_mutants_are_caught`` builds deliberately broken oracles and checks exactly that.

Paper passages: Sec. 2 (kernel, normalised frame, gradient), Sec. 3 Eq. singleSpherical and
basicdiff, Sec. 6.2 (full-cover test case).
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2507_21686_gb300.workloads import full_cover_square

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KERNELS = ["wendland_c2", "wendland_c4", "wendland_c6", "cubic_spline"]


# ---------------------------------------------------------------------------------------
# kernels as expanded polynomials in exact rationals (k(q) = sum_k b_k q^k, Sec. 2),
# written from the factored forms independently of the oracle's code
# ---------------------------------------------------------------------------------------
def _pmul(a, b):
    out = [Fr(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += Fr(x) * Fr(y)
    return out


def _ppow(a, n):
    out = [Fr(1)]
    for _ in range(n):
        out = _pmul(out, a)
    return out


ONE_MINUS_Q = [Fr(1), Fr(-1)]
PIECES = {  # list of (coefficients ascending, lo, hi)
    "wendland_c2": [(_pmul(_ppow(ONE_MINUS_Q, 4), [1, 4]), Fr(0), Fr(1))],
    "wendland_c4": [(_pmul(_ppow(ONE_MINUS_Q, 6), [1, 6, Fr(35, 3)]), Fr(0), Fr(1))],
    "wendland_c6": [(_pmul(_ppow(ONE_MINUS_Q, 8), [1, 8, 25, 32]), Fr(0), Fr(1))],
    "cubic_spline": [([Fr(1), Fr(0), Fr(-6), Fr(6)], Fr(0), Fr(1, 2)),
                     (_pmul([2], _ppow(ONE_MINUS_Q, 3)), Fr(1, 2), Fr(1))],
}


def exact_moment(kernel, p):
    """int_0^1 k(r) r^p dr, exact rational."""
    tot = Fr(0)
    for coef, lo, hi in PIECES[kernel]:
        for k, b in enumerate(coef):
            n = k + p + 1
            tot += b * (hi ** n - lo ** n) / n
    return tot


def C_times_pi(kernel):
    """Normalisation int W = 1: C = 1 / (2 pi int_0^1 k r dr)  ->  C*pi (rational)."""
    return 1 / (2 * exact_moment(kernel, 1))


def k_expanded(kernel, q):
    if q >= 1.0:
        return 0.0
    for coef, lo, hi in PIECES[kernel]:
        if float(lo) <= q < float(hi):
            return sum(float(b) * q ** k for k, b in enumerate(coef))
    return 0.0


# ---------------------------------------------------------------------------------------
# reusable checks (return the max error so mutants can be shown to fail them)
# ---------------------------------------------------------------------------------------
def full_cover_error(kernel, mutant=0):
    tris = full_cover_square(2)
    tot = sum(oracle.pair(kernel, 1.0, [0.0, 0.0], t, mutant=mutant) for t in tris)
    m20 = float(exact_moment(kernel, 3) / (2 * exact_moment(kernel, 1)))
    expect = np.zeros(16)
    expect[0] = 1.0
    expect[5] = 1.0
    expect[8] = m20
    expect[10] = m20
    return float(np.max(np.abs(tot[:15] - expect[:15])))


def wall_error(kernel, delta, mutant=0, H=1.0):
    """Particle at height delta*H above a straight wall (half-plane y <= 0 in the support)."""
    xp = np.array([0.0, delta * H])
    wall = np.array([[-3, -3, 3, -3, 3, 0], [-3, -3, 3, 0, -3, 0]], float) * H
    tot = sum(oracle.pair(kernel, H, xp, t, mutant=mutant) for t in wall)
    C = float(C_times_pi(kernel)) / math.pi
    f = lambda r: 2.0 * C * k_expanded(kernel, r) * r * math.acos(min(1.0, delta / r))
    brk = [0.5] if kernel == "cubic_spline" and delta < 0.5 else None
    g_exp, _ = integrate.quad(f, delta, 1.0, epsabs=1e-15, epsrel=1e-14, limit=200, points=brk)
    tmax = math.sqrt(max(0.0, 1.0 - delta * delta))
    h = lambda t: 2.0 * C * k_expanded(kernel, math.sqrt(delta * delta + t * t))
    brk2 = None
    if kernel == "cubic_spline" and delta < 0.5:
        brk2 = [math.sqrt(0.25 - delta * delta)]
    gr_exp, _ = integrate.quad(h, 0.0, tmax, epsabs=1e-15, epsrel=1e-14, limit=200, points=brk2)
    gr_exp = -gr_exp / H                      # points into the wall
    errs = [abs(tot[0] - g_exp), abs(tot[1]) * H, abs(tot[2] - gr_exp) * H,
            abs(tot[3]) * H, abs(tot[4] - gr_exp) * H]
    return float(max(errs))


def brute_force_error(kernel, xp, tri, H=1.0, mutant=0):
    """Cartesian 2-D adaptive quadrature over the triangle (reference-triangle map)."""
    v = np.asarray(tri, float).reshape(3, 2)
    J = abs((v[1, 0] - v[0, 0]) * (v[2, 1] - v[0, 1]) - (v[1, 1] - v[0, 1]) * (v[2, 0] - v[0, 0]))
    C = float(C_times_pi(kernel)) / math.pi

    def moment(a, b):
        def f(w, u):
            px = v[0, 0] + u * (v[1, 0] - v[0, 0]) + w * (v[2, 0] - v[0, 0])
            py = v[0, 1] + u * (v[1, 1] - v[0, 1]) + w * (v[2, 1] - v[0, 1])
            qx, qy = (px - xp[0]) / H, (py - xp[1]) / H
            return qx ** a * qy ** b * C / H ** 2 * k_expanded(kernel, math.hypot(qx, qy)) * J
        val, _ = integrate.dblquad(f, 0.0, 1.0, 0.0, lambda u: 1.0 - u, epsabs=1e-13, epsrel=1e-11)
        return val

    o = oracle.pair(kernel, H, xp, tri, mutant=mutant)
    errs = [abs(moment(0, 0) - o[0])]
    for a, b in [(1, 0), (0, 1), (2, 1), (1, 2), (0, 3)]:
        errs.append(abs(moment(a, b) - o[5 + _MIDX[(a, b)]]))
    return max(errs)


_MIDX = {(0, 0): 0, (1, 0): 1, (0, 1): 2, (2, 0): 3, (1, 1): 4, (0, 2): 5,
         (3, 0): 6, (2, 1): 7, (1, 2): 8, (0, 3): 9}


def fd_error(kernel, xp, tri, H=1.0, mutant=0, step=1e-6):
    o = oracle.pair(kernel, H, xp, tri, mutant=mutant)
    errs = []
    for ax in range(2):
        e = np.zeros(2)
        e[ax] = step * H
        gp = oracle.pair(kernel, H, np.asarray(xp) + e, tri, mutant=mutant)[0]
        gm = oracle.pair(kernel, H, np.asarray(xp) - e, tri, mutant=mutant)[0]
        fd = (gp - gm) / (2 * step * H)
        errs.append(abs(fd - o[1 + ax]) * H)
        errs.append(abs(fd - o[3 + ax]) * H)
    return max(errs)


def random_case(rng, scale=1.0):
    tri = rng.uniform(-1.2, 1.2, size=6) * scale
    xp = rng.uniform(-0.6, 0.6, size=2) * scale
    return xp, tri


# ---------------------------------------------------------------------------------------
# tests
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", KERNELS)
def test_normalisation_full_cover(kernel):
    """Sec. 6.2 first case: [-1,1]^2 in 8 triangles, x=0, h=1 -> gamma=1, grad=0; plus the
    exact second moments and vanishing odd moments of a radially symmetric kernel."""
    assert full_cover_error(kernel) < 1e-13


def test_golden_full_cover_matches_paper():
    g = json.load(open(os.path.join(GOLDEN, "full_cover_8tri.json")))
    tris = full_cover_square(2)
    for k in KERNELS:
        tot = sum(oracle.pair(k, g["h"], g["x"], t) for t in tris)
        assert abs(tot[0] - g["gamma"]) < 1e-13
        assert np.allclose(tot[1:3], g["grad_gamma"], atol=1e-13)


def test_kernel_constants_exact():
    """C in the oracle equals the exact normalisation (the paper's printed 27/(16 pi) for
    the Wendland-4 kernel does not normalise in 2-D; 9/pi does)."""
    for k in KERNELS:
        assert abs(oracle.kernel_C(k) * math.pi - float(C_times_pi(k))) < 1e-14
    assert C_times_pi("wendland_c4") == 9
    assert C_times_pi("wendland_c2") == 7
    assert C_times_pi("wendland_c6") == Fr(78, 7)
    assert C_times_pi("cubic_spline") == Fr(40, 7)
    assert abs(27 / 16 - 9) > 1   # the printed value is off by far more than rounding


@pytest.mark.parametrize("kernel", KERNELS)
def test_kernel_pointwise_matches_expansion(kernel):
    for q in np.linspace(0, 1.05, 43):
        assert abs(oracle.kernel_k(kernel, q) - k_expanded(kernel, q)) < 1e-13
        # derivative against the exact rational derivative of the expanded polynomial
        if q < 1.0 and abs(q - 0.5) > 1e-9:
            qf = Fr(float(q))
            for coef, lo, hi in PIECES[kernel]:
                if lo <= qf < hi:
                    dk = sum(k * b * qf ** (k - 1) for k, b in enumerate(coef) if k > 0)
            assert abs(oracle.kernel_dk(kernel, q) - float(dk)) < 1e-12


@pytest.mark.parametrize("kernel", KERNELS)
def test_straight_wall_through_particle(kernel):
    """gamma = 1/2 exactly and |grad| = (2/H) int_0^1 C k dq pointing into the wall."""
    H = 0.37
    assert wall_error(kernel, 0.0, H=H) < 1e-12
    tot = sum(oracle.pair(kernel, H, [0, 0], t) for t in
              np.array([[-3, -3, 3, -3, 3, 0], [-3, -3, 3, 0, -3, 0]], float) * H)
    assert abs(tot[0] - 0.5) < 1e-13
    exact = float(exact_moment(kernel, 0) / (math.pi * exact_moment(kernel, 1))) / H
    assert abs(-tot[2] - exact) * H < 1e-13


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("delta", [1e-9, 0.1, 0.4999, 0.5, 0.73, 0.999])
def test_wall_at_distance(kernel, delta):
    """1-D closed forms: gamma(d) = int_d^1 2 C k(r) r acos(d/r) dr, |grad| = line integral."""
    assert wall_error(kernel, delta) < 1e-12


def test_additivity_split_triangle():
    rng = np.random.default_rng(11)
    for k in KERNELS:
        for _ in range(6):
            xp, tri = random_case(rng)
            v = tri.reshape(3, 2)
            m = v[0] + 0.37 * (v[1] - v[0])
            t1 = np.array([v[0], m, v[2]]).ravel()
            t2 = np.array([m, v[1], v[2]]).ravel()
            a = oracle.pair(k, 1.0, xp, tri)
            b = oracle.pair(k, 1.0, xp, t1) + oracle.pair(k, 1.0, xp, t2)
            assert np.max(np.abs(a[:15] - b[:15])) < 2e-14


def test_additivity_remeshed_square():
    """The 8- and 32-triangle meshes of [-1,1]^2 give the same integrals anywhere."""
    rng = np.random.default_rng(12)
    coarse, fine = full_cover_square(2), full_cover_square(4)
    for k in KERNELS:
        for _ in range(3):
            xp = rng.uniform(-1.3, 1.3, size=2)
            a = sum(oracle.pair(k, 0.8, xp, t) for t in coarse)
            b = sum(oracle.pair(k, 0.8, xp, t) for t in fine)
            assert np.max(np.abs(a[:15] - b[:15])) < 5e-14


def _transform_moments(M, R):
    """Moments of the rotated field: M'_{ab} = int (R p)_x^a (R p)_y^b W (tensor transform)."""
    out = np.zeros(10)
    for (a, b), idx in _MIDX.items():
        # expand (r00 x + r01 y)^a (r10 x + r11 y)^b into monomials
        poly = {(0, 0): 1.0}
        for _ in range(a):
            poly = _mono_mul(poly, {(1, 0): R[0, 0], (0, 1): R[0, 1]})
        for _ in range(b):
            poly = _mono_mul(poly, {(1, 0): R[1, 0], (0, 1): R[1, 1]})
        out[idx] = sum(c * M[_MIDX[e]] for e, c in poly.items())
    return out


def _mono_mul(p, q):
    out = {}
    for (i, j), c in p.items():
        for (k, l), d in q.items():
            out[(i + k, j + l)] = out.get((i + k, j + l), 0.0) + c * d
    return out


@pytest.mark.parametrize("reflect", [False, True])
def test_rigid_motion_and_reflection(reflect):
    rng = np.random.default_rng(13 + reflect)
    for k in KERNELS:
        xp, tri = random_case(rng)
        a = rng.uniform(0, 2 * math.pi)
        R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
        if reflect:
            R = R @ np.diag([1.0, -1.0])
        t = rng.uniform(-5, 5, size=2)
        xp2 = R @ xp + t
        tri2 = (tri.reshape(3, 2) @ R.T + t).ravel()
        o1 = oracle.pair(k, 1.0, xp, tri)
        o2 = oracle.pair(k, 1.0, xp2, tri2)
        assert abs(o1[0] - o2[0]) < 1e-13
        assert np.allclose(R @ o1[1:3], o2[1:3], atol=1e-13)
        assert np.allclose(R @ o1[3:5], o2[3:5], atol=1e-13)
        assert np.allclose(_transform_moments(o1[5:15], R), o2[5:15], atol=1e-13)


def test_scale_invariance_and_orientation():
    rng = np.random.default_rng(14)
    for k in KERNELS:
        xp, tri = random_case(rng)
        lam = 3.7
        o1 = oracle.pair(k, 1.0, xp, tri)
        o2 = oracle.pair(k, lam, lam * xp, lam * tri)
        assert abs(o1[0] - o2[0]) < 1e-13
        assert np.allclose(o1[1:5] / lam, o2[1:5], atol=1e-13)
        assert np.allclose(o1[5:15], o2[5:15], atol=1e-13)
        cw = tri.reshape(3, 2)[[0, 2, 1]].ravel()
        o3 = oracle.pair(k, 1.0, xp, cw)
        assert np.max(np.abs(o1[:15] - o3[:15])) < 1e-14
        deg = np.array([0.125, 0.25, 0.25, 0.5, 0.5, 1.0])   # exactly collinear
        assert np.all(oracle.pair(k, 1.0, [0.0, 0.0], deg)[:15] == 0.0)
        dup = np.array([0.125, 0.25, 0.125, 0.25, 0.5, -0.5])  # two coincident vertices
        assert np.all(oracle.pair(k, 1.0, [0.0, 0.0], dup)[:15] == 0.0)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(15)
    for k in KERNELS:
        for _ in range(3):
            xp, tri = random_case(rng)
            assert fd_error(k, xp, tri) < 5e-8


def test_vertex_gradient_translation_identity_and_fd():
    rng = np.random.default_rng(16)
    for k in KERNELS:
        for _ in range(3):
            xp, tri = random_case(rng)
            vg = oracle.vertex_grad(k, 1.0, xp, tri)
            o = oracle.pair(k, 1.0, xp, tri)
            assert np.allclose(vg.sum(axis=0), -o[1:3], atol=1e-13)
            h = 1e-6
            for j in range(6):
                e = np.zeros(6)
                e[j] = h
                fd = (oracle.pair(k, 1.0, xp, tri + e)[0] - oracle.pair(k, 1.0, xp, tri - e)[0]) / (2 * h)
                assert abs(fd - vg.ravel()[j]) < 5e-8


@pytest.mark.parametrize("kernel", KERNELS)
def test_brute_force_2d_quadrature(kernel):
    """Small triangles partly inside the support: oracle vs Cartesian dblquad."""
    rng = np.random.default_rng(17)
    for _ in range(2):
        c = rng.uniform(-0.9, 0.9, size=2)
        tri = (c + rng.uniform(-0.35, 0.35, size=(3, 2))).ravel()
        assert brute_force_error(kernel, np.zeros(2), tri) < 1e-10


def _exact_keep(px, py, tri, H):
    """Exact rational distance test: closed triangle within distance < H."""
    P = (Fr(float(px)), Fr(float(py)))
    V = [(Fr(float(tri[2 * j])), Fr(float(tri[2 * j + 1]))) for j in range(3)]
    crs = []
    best = None
    for e in range(3):
        a, b = V[e], V[(e + 1) % 3]
        ex, ey = b[0] - a[0], b[1] - a[1]
        wx, wy = P[0] - a[0], P[1] - a[1]
        crs.append(wx * ey - wy * ex)
        l2 = ex * ex + ey * ey
        t = (wx * ex + wy * ey) / l2 if l2 else Fr(0)
        t = min(max(t, Fr(0)), Fr(1))
        dx, dy = wx - t * ex, wy - t * ey
        d2 = dx * dx + dy * dy
        best = d2 if best is None else min(best, d2)
    if any(c != 0 for c in crs) and (all(c >= 0 for c in crs) or all(c <= 0 for c in crs)):
        return True, Fr(0)
    return best < Fr(H) * Fr(H), best


def test_cull_matches_exact_rational_predicate():
    rng = np.random.default_rng(18)
    parts = np.zeros((300, 4), np.float32)
    parts[:, :2] = rng.uniform(0, 1, size=(300, 2)).astype(np.float32)
    tris = rng.uniform(0, 1, size=(60, 6)).astype(np.float32)
    tris[:20] = (tris[:20] - 0.5) * 0.1 + tris[:20, :2].repeat(3, axis=0).reshape(20, 6)
    # zero-area triangles: a segment with a repeated vertex, and three collinear vertices
    tris[20] = [0.5, 0.0, 0.5, 0.0, 0.5, 0.5]
    tris[21] = [0.125, 0.25, 0.25, 0.5, 0.5, 1.0]
    parts[:4, :2] = [[0.5, 0.9], [0.5, 0.55], [0.625, 1.25], [0.0625, 0.125]]   # on those lines
    H = 0.0625
    off, pt = oracle.cull(parts, tris, H)
    got = set()
    for i in range(len(parts)):
        for q in range(off[i], off[i + 1]):
            got.add((i, int(pt[q])))
        assert list(pt[off[i]:off[i + 1]]) == sorted(pt[off[i]:off[i + 1]])
    want = set()
    H2 = Fr(H) * Fr(H)
    for i in range(len(parts)):
        for t in range(len(tris)):
            keep, d2 = _exact_keep(parts[i, 0], parts[i, 1], tris[t], H)
            if keep and d2 != 0 and abs(d2 - H2) < Fr(1, 10 ** 12):
                continue                       # ties at the threshold are rounding-defined
            if keep:
                want.add((i, t))
    near = {(i, t) for (i, t) in got - want
            if abs(_exact_keep(parts[i, 0], parts[i, 1], tris[t], H)[1] - H2) < Fr(1, 10 ** 12)}
    assert got - near == want


def test_quadrature_nodes_against_numpy():
    x, w = oracle.gauss_legendre(20)
    xr, wr = np.polynomial.legendre.leggauss(20)
    assert np.allclose(np.sort(x), np.sort(xr), atol=1e-15)
    assert np.allclose(w[np.argsort(x)], wr[np.argsort(xr)], atol=1e-14)


# ---------------------------------------------------------------------------------------
# each plausible mistake, planted in the oracle on the CPU, fails a pin
# ---------------------------------------------------------------------------------------
def test_mutants_are_caught():
    rng = np.random.default_rng(19)
    xp, tri = np.zeros(2), np.array([0.2, -0.1, 0.9, 0.3, 0.1, 0.7])
    # 1: wrong normalisation constant (the printed Wendland constant applied to C2)
    assert full_cover_error("wendland_c2", mutant=1) > 1e-3
    # 2: gradient sign flip
    assert wall_error("wendland_c2", 0.3, mutant=2) > 1e-3
    assert fd_error("wendland_c2", xp, tri, mutant=2) > 1e-3
    # 3: transposed moment exponents (M21 <-> M12, M10 <-> M01 ...)
    assert brute_force_error("wendland_c2", xp, tri, mutant=3) > 1e-4
    # 4: polar Jacobian r dropped
    assert full_cover_error("wendland_c2", mutant=4) > 1e-3
    # the unmutated oracle passes the same checks
    assert full_cover_error("wendland_c2") < 1e-13
    assert brute_force_error("wendland_c2", xp, tri) < 1e-10
    del rng
