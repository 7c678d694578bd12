"""FP64 numpy reference for the learned surrogate (a component the paper does not have).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s CPU legs, never by the
product path, and it imports nothing from the product path.

What it restates, in plain array code:
  * the canonical frame of a pair (particle frame with H = 1): rotate the triangle so that
    its centroid lies on +x, reflect y -> -y if its vertex closest to the particle then lies
    below the axis, list the vertices counter-clockwise from that closest one (lowest index
    on ties), and the guard that decides whether the network may be used;
  * the network 6 -> 64 -> 64 -> 64 -> 3 with the tanh form of GELU between layers, its
    loss (1/B) sum_rows sum_c w_c (y_c - t_c)^2 and that loss's gradient by backpropagation;
  * optional emulation of the tensor-core operand roundings (float64 -> float32 -> operand
    type, round to nearest even): forward products take FP16 operands and the GELU between
    them is evaluated step by step in FP16 as the GPU does, backward products take BF16
    operands, so that GPU and reference differ only in accumulation order and in the GPU's
    hardware tanh approximation.
Parameter layout (flat float): W1[64][6] b1[64] W2[64][64] b2[64] W3[64][64] b3[64]
W4[3][64] b4[3], W[out][in].

Pins (tests/test_oracle_surrogate_pins.py): central finite differences of the loss against the
backpropagated gradient; invariance of the canonical inputs under rotation, reflection and
relabelling of the triangle; the inverse transform reproducing the input triangle; the
network reducing to its output bias when all weights are zero.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_OUT = 6, 64, 3
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_OUT, N_HID)), ("b4", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)      # 8963

MIN_SIZE, MAX_SIZE = 0.1, 0.45
MIN_CENTROID, MAX_RADIUS = 0.3, 1.5
SIN_MIN_ANGLE = math.sin(math.radians(15.0))

GELU_K = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def unpack(flat):
    """Flat parameter vector -> dict of float64 arrays."""
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(x):
    """Round to bfloat16 (via float32, round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def f16(x):
    """Round to IEEE half (via float32, round to nearest even), returned as float64."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def _exact(a):
    return np.asarray(a, dtype=np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_K * (z + GELU_A * z ** 3)))


def gelu_f16(z):
    """The GELU as the GPU evaluates it on FP16 pairs: z rounded to FP16, then
    u = (z*z rounded) * ka + k (one rounding, a fused multiply-add), u = u * z (rounded),
    t = tanh(u) rounded (the GPU's hardware approximation is within about one FP16 step of
    it), h = z / 2, result = h * t + h (one rounding).  Products of FP16 values are exact in
    float64, so each rounded step is one rounding of the exact value."""
    K = f16(GELU_K)
    KA = f16(np.float32(GELU_K) * np.float32(GELU_A))
    with np.errstate(over="ignore", invalid="ignore"):
        z = f16(z)
        u = f16(f16(f16(z * z) * KA + K) * z)
        t = f16(np.tanh(u))
        h = f16(0.5 * z)
        return f16(h * t + h)


def gelu_grad(z):
    u = GELU_K * (z + GELU_A * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_K * (1.0 + 3.0 * GELU_A * z * z)


# ---------------------------------------------------------------------------------------
# canonical frame and guard
# ---------------------------------------------------------------------------------------
def canonicalize(local):
    """local [P, 6] triangles in the particle frame (H = 1) -> dict with
    x [P, 6] canonical vertices, cs, sn (rotation taking the centroid direction to +x),
    refl (+1 / -1), area, and the guard quantities lmax, smin, rc, rmax, accept."""
    v = np.asarray(local, dtype=np.float64).reshape(-1, 3, 2)
    c = v.mean(axis=1)
    r = np.hypot(c[:, 0], c[:, 1])
    safe = r > 0
    cs = np.where(safe, c[:, 0] / np.where(safe, r, 1.0), 1.0)
    sn = np.where(safe, c[:, 1] / np.where(safe, r, 1.0), 0.0)
    # rotation by -angle(centroid): (x, y) -> (cs x + sn y, -sn x + cs y)
    q = np.empty_like(v)
    q[..., 0] = cs[:, None] * v[..., 0] + sn[:, None] * v[..., 1]
    q[..., 1] = -sn[:, None] * v[..., 0] + cs[:, None] * v[..., 1]
    cr = (q[:, 1, 0] - q[:, 0, 0]) * (q[:, 2, 1] - q[:, 0, 1]) - \
         (q[:, 1, 1] - q[:, 0, 1]) * (q[:, 2, 0] - q[:, 0, 0])
    d = q[..., 0] ** 2 + q[..., 1] ** 2
    k = np.argmin(d, axis=1)                     # first minimum: lowest index on ties
    rows = np.arange(len(q))
    # mirror y -> -y when the closest vertex lies below the axis
    refl = np.where(q[rows, k, 1] < 0, -1.0, 1.0)
    q[..., 1] *= refl[:, None]
    # counter-clockwise from the closest vertex: forward if the mirrored labelled order is
    # counter-clockwise, backward otherwise
    step = np.where(refl * cr < 0, 2, 1)
    idx = (k[:, None] + step[:, None] * np.arange(3)[None, :]) % 3
    x = np.take_along_axis(q, idx[:, :, None], axis=1)
    area = 0.5 * np.abs(cr)
    e = np.roll(x, -1, axis=1) - x               # edges v0v1, v1v2, v2v0
    ln = np.hypot(e[..., 0], e[..., 1])
    lmax = ln.max(axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        s0 = 2 * area / (ln[:, 0] * ln[:, 2])
        s1 = 2 * area / (ln[:, 0] * ln[:, 1])
        s2 = 2 * area / (ln[:, 1] * ln[:, 2])
    smin = np.nan_to_num(np.minimum(np.minimum(s0, s1), s2), nan=0.0)
    rmax = np.sqrt(d.max(axis=1))
    accept = (area > 0) & (lmax >= MIN_SIZE) & (lmax <= MAX_SIZE) & (smin >= SIN_MIN_ANGLE) & \
             (r >= MIN_CENTROID) & (rmax <= MAX_RADIUS)
    return dict(x=x.reshape(-1, 6), cs=cs, sn=sn, refl=refl, area=area, lmax=lmax, smin=smin,
                rc=r, rmax=rmax, accept=accept)


def guard_margin(cn):
    """Smallest relative distance of any guard quantity to its threshold (pairs closer than
    a few FP32 roundings may be decided differently by FP32 and FP64 arithmetic)."""
    rel = lambda a, t: np.abs(a - t) / t
    return np.minimum.reduce([rel(cn["lmax"], MIN_SIZE), rel(cn["lmax"], MAX_SIZE),
                              rel(cn["smin"], SIN_MIN_ANGLE), rel(cn["rc"], MIN_CENTROID),
                              rel(cn["rmax"], MAX_RADIUS)])


def frame_margin(cn):
    """How far the discrete choices of the canonical frame are from a tie: the relative gap
    between the two smallest vertex distances and |y| of the closest vertex (both in units
    of the triangle's size).  Near zero, FP32 and FP64 may pick different (equally valid)
    frames."""
    x = cn["x"].reshape(-1, 3, 2)
    d = np.sort(np.hypot(x[..., 0], x[..., 1]), axis=1)
    return np.minimum((d[:, 1] - d[:, 0]) / cn["lmax"], np.abs(x[:, 0, 1]) / cn["lmax"])


def uncanonicalize_grad(cn, g):
    """canonical gradient [P, 2] -> particle-frame gradient (inverse reflection, rotation)."""
    gx, gy = g[:, 0], cn["refl"] * g[:, 1]
    return np.stack([cn["cs"] * gx - cn["sn"] * gy, cn["sn"] * gx + cn["cs"] * gy], axis=1)


def canonical_targets(cn, gamma, grad_local):
    """training targets: (gamma, canonical local-frame gradient) / area."""
    gx, gy = grad_local[:, 0], grad_local[:, 1]
    gxc = cn["cs"] * gx + cn["sn"] * gy
    gyc = cn["refl"] * (-cn["sn"] * gx + cn["cs"] * gy)
    a = cn["area"]
    return np.stack([gamma / a, gxc / a, gyc / a], axis=1)


# ---------------------------------------------------------------------------------------
# network, loss, gradient
# ---------------------------------------------------------------------------------------
def forward(params, X, emulate_tc=False):
    """X [B, 6] -> (Y [B, 3], cache)."""
    p = unpack(params)
    rnd = f16 if emulate_tc else _exact
    act = gelu_f16 if emulate_tc else gelu
    H0 = np.asarray(X, dtype=np.float64)
    Z1 = rnd(H0) @ rnd(p["W1"]).T + p["b1"]
    H1 = act(Z1)
    Z2 = rnd(H1) @ rnd(p["W2"]).T + p["b2"]
    H2 = act(Z2)
    Z3 = rnd(H2) @ rnd(p["W3"]).T + p["b3"]
    H3 = act(Z3)
    Y = rnd(H3) @ rnd(p["W4"]).T + p["b4"]
    return Y, dict(H0=H0, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Z3=Z3, H3=H3)


def loss(params, X, T, w, emulate_tc=False):
    Y, _ = forward(params, X, emulate_tc)
    return float(np.mean(np.sum(np.asarray(w)[None, :] * (Y - T) ** 2, axis=1)))


def loss_and_grad(params, X, T, w, emulate_tc=False):
    """(loss, flat gradient) by backpropagation through the four layers."""
    p = unpack(params)
    rnd = bf16 if emulate_tc else _exact
    Y, k = forward(params, X, emulate_tc)
    B = Y.shape[0]
    w = np.asarray(w, dtype=np.float64)
    D = Y - T
    L = float(np.mean(np.sum(w[None, :] * D ** 2, axis=1)))
    dY = 2.0 * w[None, :] * D / B
    g = {}
    g["W4"] = rnd(dY).T @ rnd(k["H3"])
    g["b4"] = dY.sum(axis=0)
    dZ3 = (rnd(dY) @ rnd(p["W4"])) * gelu_grad(k["Z3"])
    g["W3"] = rnd(dZ3).T @ rnd(k["H2"])
    g["b3"] = dZ3.sum(axis=0)
    dZ2 = (rnd(dZ3) @ rnd(p["W3"])) * gelu_grad(k["Z2"])
    g["W2"] = rnd(dZ2).T @ rnd(k["H1"])
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (rnd(dZ2) @ rnd(p["W2"])) * gelu_grad(k["Z1"])
    g["W1"] = rnd(dZ1).T @ rnd(k["H0"])
    g["b1"] = dZ1.sum(axis=0)
    return L, pack(g)


def loss_weights(C):
    """per-output weights 1/scale^2: the averaged kernel is at most C, its gradient ~2C."""
    return np.array([1.0 / C ** 2, 1.0 / (4 * C ** 2), 1.0 / (4 * C ** 2)])


def surrogate_local(params, local, emulate_tc=True):
    """Network prediction for particle-frame pairs (H = 1): (gamma, local-frame gradient)
    [P, 3] and the guard result; rows the guard rejects are NaN (the analytic path's)."""
    cn = canonicalize(local)
    Y, _ = forward(params, cn["x"], emulate_tc)
    a = cn["area"][:, None]
    g = uncanonicalize_grad(cn, a * Y[:, 1:3])
    out = np.concatenate([a * Y[:, :1], g], axis=1)
    out[~cn["accept"]] = np.nan
    return out, cn
