"""FP64 CPU oracle for the 2-D analytic SPH boundary integrals (arXiv 2507.21686).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product path (``paper_2507_21686_gb300``) never
imports it, and it never imports the product path.  It computes every result from the
plain definition (Sec. 2 Eq. sphintegral / nablaIntegral, Sec. 3 Eq. singleSpherical) by
quadrature, in ``sph2d_oracle.c``; this module only builds and marshals.

``pair_field`` / ``pairs_field`` / ``particle_field_sums``: piecewise-linear boundary fields
(Sec. 3, Eq. singleSpherical and basicdiff) by polar quadrature of the barycentric field times
W and grad W.  ``pair_field_p`` / ``pairs_field_p`` / ``particle_field_sums_p``: Lagrange
fields of order 1-3 from node values (``field_nodes`` gives the node positions), by the same
quadrature with the field evaluated from its nodal basis.

Outputs of ``pairs`` (per pair, 16 doubles):
  0 gamma | 1,2 grad gamma (divergence theorem) | 3,4 grad gamma (polar route, k')
  5..14 moments M00 M10 M01 M20 M11 M02 M30 M21 M12 M03 | 15 quadrature flag
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph2d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

KERNEL_IDS = {"wendland_c2": 0, "wendland_c4": 1, "wendland_c6": 2, "cubic_spline": 3}

_libs: dict[int, ctypes.CDLL] = {}


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction).  ``mutant`` > 0 builds a
    deliberately wrong variant used by the pin tests to show each pin has teeth."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           f"-DORC_MUTANT={mutant}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(mutant: int = 0) -> ctypes.CDLL:
    if mutant in _libs:
        return _libs[mutant]
    lib = ctypes.CDLL(build(mutant))
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    D = ctypes.c_double
    Ci = ctypes.c_int
    lib.orc_pair.argtypes = [Ci, D, P, P, P]
    lib.orc_vertex_grad.argtypes = [Ci, D, P, P, P]
    lib.orc_cull.argtypes = [P, I64, Ci, P, I64, D, P, P, P]
    lib.orc_particle_sums.argtypes = [Ci, D, P, I64, Ci, P, P, P, Ci, P, P, P, P]
    lib.orc_pairs.argtypes = [Ci, D, P, I64, P]
    lib.orc_pairs_vertex_grad.argtypes = [Ci, D, P, I64, P]
    lib.orc_pair_field.argtypes = [Ci, D, P, P, P, P]
    lib.orc_grad_jacobian.argtypes = [Ci, D, P, P, P]
    lib.orc_pairs_grad_jacobian.argtypes = [Ci, D, P, I64, P]
    lib.orc_pairs_field.argtypes = [Ci, D, P, P, I64, P]
    lib.orc_pair_field_p.argtypes = [Ci, D, P, P, Ci, P, P]
    lib.orc_pairs_field_p.argtypes = [Ci, D, P, Ci, P, I64, P]
    lib.orc_field_nodes.argtypes = [P, Ci, P]
    lib.orc_kernel_C.argtypes = [Ci]
    lib.orc_kernel_C.restype = D
    lib.orc_kernel_k.argtypes = [Ci, D]
    lib.orc_kernel_k.restype = D
    lib.orc_kernel_dk.argtypes = [Ci, D]
    lib.orc_kernel_dk.restype = D
    lib.orc_gauss_legendre.argtypes = [Ci, P, P]
    for f in ("orc_pair", "orc_vertex_grad", "orc_cull", "orc_particle_sums", "orc_pairs",
              "orc_pairs_vertex_grad", "orc_num_threads", "orc_version", "orc_pair_field",
              "orc_pairs_field", "orc_grad_jacobian", "orc_pairs_grad_jacobian", "orc_pair_field_p",
              "orc_pairs_field_p", "orc_field_nodes"):
        getattr(lib, f).restype = ctypes.c_int if f != "orc_kernel_C" else D
    _libs[mutant] = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _kid(kernel) -> int:
    return KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel)


def num_threads() -> int:
    return _lib().orc_num_threads()


def kernel_C(kernel, mutant: int = 0) -> float:
    return _lib(mutant).orc_kernel_C(_kid(kernel))


def kernel_k(kernel, q: float) -> float:
    return _lib().orc_kernel_k(_kid(kernel), float(q))


def kernel_dk(kernel, q: float) -> float:
    return _lib().orc_kernel_dk(_kid(kernel), float(q))


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _lib().orc_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def pair(kernel, H: float, xp, tri, mutant: int = 0) -> np.ndarray:
    """One (particle, triangle) pair in world units -> 16 doubles (layout in module doc)."""
    xp = np.ascontiguousarray(xp, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.float64).reshape(6)
    out = np.zeros(16)
    rc = _lib(mutant).orc_pair(_kid(kernel), float(H), _ptr(xp), _ptr(tri), _ptr(out))
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return out


def pairs(kernel, H: float, pairs_arr: np.ndarray, mutant: int = 0) -> np.ndarray:
    """Many pairs [P, 8] (px, py, x0, y0, x1, y1, x2, y2) -> [P, 16]."""
    p = np.ascontiguousarray(pairs_arr, dtype=np.float64).reshape(-1, 8)
    out = np.zeros((len(p), 16))
    rc = _lib(mutant).orc_pairs(_kid(kernel), float(H), _ptr(p), len(p), _ptr(out))
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return out


def vertex_grad(kernel, H: float, xp, tri) -> np.ndarray:
    """d gamma / d vertex, [3, 2], by the transport theorem (edge line integrals)."""
    xp = np.ascontiguousarray(xp, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.float64).reshape(6)
    out = np.zeros(6)
    _lib().orc_vertex_grad(_kid(kernel), float(H), _ptr(xp), _ptr(tri), _ptr(out))
    return out.reshape(3, 2)


def pairs_vertex_grad(kernel, H: float, pairs_arr: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(pairs_arr, dtype=np.float64).reshape(-1, 8)
    out = np.zeros((len(p), 6))
    _lib().orc_pairs_vertex_grad(_kid(kernel), float(H), _ptr(p), len(p), _ptr(out))
    return out


def pair_field(kernel, H: float, xp, tri, values, mutant: int = 0) -> np.ndarray:
    """Linear boundary field on one triangle (vertex values [3], caller's vertex order) ->
    [<A>, <grad A>_x, <grad A>_y] by polar quadrature of the field times W and grad W."""
    xp = np.ascontiguousarray(xp, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.float64).reshape(6)
    a = np.ascontiguousarray(values, dtype=np.float64).reshape(3)
    out = np.zeros(3)
    rc = _lib(mutant).orc_pair_field(_kid(kernel), float(H), _ptr(xp), _ptr(tri), _ptr(a), _ptr(out))
    if rc < 0:
        raise ValueError("oracle: bad arguments")
    return out


def pairs_field(kernel, H: float, pairs_arr: np.ndarray, values: np.ndarray, mutant: int = 0) -> np.ndarray:
    """Many pairs [P, 8] with vertex values [P, 3] -> [P, 3] (<A>, <grad A>)."""
    p = np.ascontiguousarray(pairs_arr, dtype=np.float64).reshape(-1, 8)
    a = np.ascontiguousarray(values, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((len(p), 3))
    rc = _lib(mutant).orc_pairs_field(_kid(kernel), float(H), _ptr(p), _ptr(a), len(p), _ptr(out))
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return out


def nodes_per_triangle(order: int) -> int:
    return (order + 1) * (order + 2) // 2


def field_nodes(triangles: np.ndarray, order: int) -> np.ndarray:
    """World positions of the order-k Lagrange nodes of each triangle: [M, nn, 2]."""
    tris = np.ascontiguousarray(triangles, dtype=np.float64).reshape(-1, 6)
    nn = nodes_per_triangle(order)
    out = np.zeros((len(tris), nn, 2))
    lib = _lib()
    for m in range(len(tris)):
        row = np.ascontiguousarray(tris[m])
        buf = np.zeros(2 * nn)
        if lib.orc_field_nodes(_ptr(row), int(order), _ptr(buf)) != 0:
            raise ValueError("oracle: bad order")
        out[m] = buf.reshape(nn, 2)
    return out


def pair_field_p(kernel, H: float, xp, tri, order: int, values, mutant: int = 0) -> np.ndarray:
    """Lagrange field of order 1-3 on one triangle (node values [nn]) -> [<A>, <grad A>]."""
    xp = np.ascontiguousarray(xp, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.float64).reshape(6)
    a = np.ascontiguousarray(values, dtype=np.float64).reshape(nodes_per_triangle(order))
    out = np.zeros(3)
    rc = _lib(mutant).orc_pair_field_p(_kid(kernel), float(H), _ptr(xp), _ptr(tri), int(order), _ptr(a), _ptr(out))
    if rc < 0:
        raise ValueError("oracle: bad arguments")
    return out


def pairs_field_p(kernel, H: float, pairs_arr: np.ndarray, order: int, values: np.ndarray,
                  mutant: int = 0) -> np.ndarray:
    """Many pairs [P, 8] with node values [P, nn] -> [P, 3] (<A>, <grad A>)."""
    p = np.ascontiguousarray(pairs_arr, dtype=np.float64).reshape(-1, 8)
    a = np.ascontiguousarray(values, dtype=np.float64).reshape(-1, nodes_per_triangle(order))
    out = np.zeros((len(p), 3))
    rc = _lib(mutant).orc_pairs_field_p(_kid(kernel), float(H), _ptr(p), int(order), _ptr(a), len(p), _ptr(out))
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return out


def particle_field_sums_p(kernel, H: float, particles: np.ndarray, triangles: np.ndarray, off, pair_tri,
                          order: int, node_values: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per-particle sums of Lagrange fields of order 1-3: node_values [M, nn, nf] ->
    value [N, nf], grad [N, nf, 2]."""
    parts = np.asarray(particles, dtype=np.float32)
    tris = np.asarray(triangles, dtype=np.float32).reshape(-1, 6)
    nv = np.asarray(node_values, dtype=np.float32)
    if nv.ndim == 2:
        nv = nv[:, :, None]
    nf = nv.shape[2]
    off = np.asarray(off, dtype=np.int64)
    pt = np.asarray(pair_tri, dtype=np.int64)
    pid = np.repeat(np.arange(len(parts)), np.diff(off))
    pr = np.zeros((len(pt), 8))
    pr[:, :2] = parts[pid, :2]
    pr[:, 2:] = tris[pt]
    val = np.zeros((len(parts), nf))
    grad = np.zeros((len(parts), nf, 2))
    for f in range(nf):
        r = pairs_field_p(kernel, H, pr, order, nv[pt, :, f].astype(np.float64))
        np.add.at(val[:, f], pid, r[:, 0])
        np.add.at(grad[:, f, 0], pid, r[:, 1])
        np.add.at(grad[:, f, 1], pid, r[:, 2])
    return val, grad


def particle_field_sums(kernel, H: float, particles: np.ndarray, triangles: np.ndarray, off, pair_tri,
                        vertex_values: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per-particle sums of linear boundary fields: vertex_values [M, 3, nf] ->
    value [N, nf], grad [N, nf, 2] (pairs in ascending triangle id per particle)."""
    parts = np.asarray(particles, dtype=np.float32)
    tris = np.asarray(triangles, dtype=np.float32).reshape(-1, 6)
    vv = np.asarray(vertex_values, dtype=np.float32)
    if vv.ndim == 2:
        vv = vv[:, :, None]
    nf = vv.shape[2]
    off = np.asarray(off, dtype=np.int64)
    pt = np.asarray(pair_tri, dtype=np.int64)
    pid = np.repeat(np.arange(len(parts)), np.diff(off))
    pr = np.zeros((len(pt), 8))
    pr[:, :2] = parts[pid, :2]
    pr[:, 2:] = tris[pt]
    val = np.zeros((len(parts), nf))
    grad = np.zeros((len(parts), nf, 2))
    for f in range(nf):
        r = pairs_field(kernel, H, pr, vv[pt, :, f].astype(np.float64))
        np.add.at(val[:, f], pid, r[:, 0])
        np.add.at(grad[:, f, 0], pid, r[:, 1])
        np.add.at(grad[:, f, 1], pid, r[:, 2])
    return val, grad


def grad_jacobian(kernel, H: float, xp, tri) -> np.ndarray:
    """d grad gamma / d nu_j, [3, 2, 2] with [j, b, a] = d (grad gamma)_b / d (nu_j)_a, from the
    divergence-theorem boundary form differentiated edge by edge (1-D quadratures)."""
    xp = np.ascontiguousarray(xp, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.float64).reshape(6)
    out = np.zeros(12)
    _lib().orc_grad_jacobian(_kid(kernel), float(H), _ptr(xp), _ptr(tri), _ptr(out))
    return out.reshape(3, 2, 2)


def pairs_grad_jacobian(kernel, H: float, pairs_arr: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(pairs_arr, dtype=np.float64).reshape(-1, 8)
    out = np.zeros((len(p), 12))
    _lib().orc_pairs_grad_jacobian(_kid(kernel), float(H), _ptr(p), len(p), _ptr(out))
    return out.reshape(-1, 3, 2, 2)


def cull(particles: np.ndarray, triangles: np.ndarray, H: float):
    """Brute-force pair list: (off int64 [N+1], tri int32 [P]), ascending triangle ids."""
    parts = np.ascontiguousarray(particles, dtype=np.float32)
    stride = parts.shape[1]
    tris = np.ascontiguousarray(triangles, dtype=np.float32).reshape(-1, 6)
    n = len(parts)
    counts = np.zeros(n, dtype=np.int64)
    lib = _lib()
    rc = lib.orc_cull(_ptr(parts), n, stride, _ptr(tris), len(tris), float(H), _ptr(counts), None, None)
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    out = np.zeros(int(off[-1]), dtype=np.int32)
    lib.orc_cull(_ptr(parts), n, stride, _ptr(tris), len(tris), float(H), None, _ptr(off), _ptr(out))
    return off, out


def particle_sums(kernel, H: float, particles: np.ndarray, triangles: np.ndarray, off, pair_tri,
                  moment_degree: int = -1):
    """Per-particle sums gamma [N], grad [N,2], moments [N,nm], quadrature flags [N]."""
    parts = np.ascontiguousarray(particles, dtype=np.float32)
    tris = np.ascontiguousarray(triangles, dtype=np.float32).reshape(-1, 6)
    off = np.ascontiguousarray(off, dtype=np.int64)
    pt = np.ascontiguousarray(pair_tri, dtype=np.int32)
    n = len(parts)
    nm = 0 if moment_degree < 0 else (moment_degree + 1) * (moment_degree + 2) // 2
    g = np.zeros(n)
    gr = np.zeros((n, 2))
    mom = np.zeros((n, max(nm, 1)))
    fl = np.zeros(n, dtype=np.int32)
    rc = _lib().orc_particle_sums(_kid(kernel), float(H), _ptr(parts), n, parts.shape[1], _ptr(tris),
                                  _ptr(off), _ptr(pt), int(moment_degree), _ptr(g), _ptr(gr),
                                  _ptr(mom), _ptr(fl))
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return g, gr, mom[:, :nm], fl
