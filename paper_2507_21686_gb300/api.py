"""Python API over libsph2d: PyTorch supplies device memory and streams; every step of the
computation runs in the library's CUDA kernels.

    from paper_2507_21686_gb300 import boundary_integrals
    gamma, grad_gamma, moments = boundary_integrals(particles, tris, "wendland_c2", H,
                                                    moment_degree=3, mode="fp32_fixup")

particles: float32 [N, 4] (x, y, 0, 0) or [N, 2]; tris: float32 [M, 6] or [M, 3, 2].  CUDA
tensors are used in place; CPU tensors are copied to the device (and results copied back).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import KERNELS, MODES, Stats, check


def _kernel_id(kernel) -> int:
    if isinstance(kernel, str):
        if kernel not in KERNELS:
            raise ValueError(f"unknown kernel {kernel!r}; expected one of {sorted(KERNELS)}")
        return KERNELS[kernel]
    return int(kernel)


def _mode_id(mode) -> int:
    if isinstance(mode, str):
        if mode not in MODES:
            raise ValueError(f"unknown mode {mode!r}; expected one of {sorted(MODES)}")
        return MODES[mode]
    return int(mode)


def num_moments(deg: int) -> int:
    return 0 if deg < 0 else (deg + 1) * (deg + 2) // 2


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def as_particles(p: torch.Tensor, device) -> torch.Tensor:
    """float32 [N, 4] contiguous on `device` (pads [N, 2] with zeros)."""
    if p.dim() != 2 or p.shape[1] not in (2, 4):
        raise ValueError("particles must be [N, 2] or [N, 4]")
    if p.shape[1] == 2:
        q = torch.zeros((p.shape[0], 4), dtype=torch.float32, device=p.device)
        q[:, :2] = p
        p = q
    return p.to(device=device, dtype=torch.float32, non_blocking=True).contiguous()


def as_triangles(t: torch.Tensor, device) -> torch.Tensor:
    if t.dim() == 3:
        t = t.reshape(t.shape[0], 6)
    if t.dim() != 2 or t.shape[1] != 6:
        raise ValueError("triangles must be [M, 6] or [M, 3, 2]")
    return t.to(device=device, dtype=torch.float32, non_blocking=True).contiguous()


class Context:
    """One libsph2d context (scratch memory + culling state) on one CUDA device."""

    def __init__(self, device: int | None = None):
        self.lib = _lib.load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        st = self.lib.sph2d_init(ctypes.byref(h), self.device, None)
        if st != 0:
            raise _lib.Sph2dError(st, "sph2d_init failed")
        self.h = h
        self._builds = 0          # pair-list builds so far (a backward can reuse the latest)

    def close(self):
        if getattr(self, "h", None):
            self.lib.sph2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _bind_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        check(self.lib, self.h, self.lib.sph2d_set_stream(self.h, ctypes.c_void_p(s)))

    def _dev(self):
        return torch.device("cuda", self.device)

    # -- culling ------------------------------------------------------------------------
    def build_cells(self, particles, tris, H: float):
        p = as_particles(particles, self._dev())
        t = as_triangles(tris, self._dev())
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_build_cells(self.h, _ptr(p), p.shape[0], _ptr(t),
                                                            t.shape[0], float(H)))
        self._keep = (p, t)
        self._builds += 1
        return self

    def pair_count(self) -> int:
        n = ctypes.c_int64()
        check(self.lib, self.h, self.lib.sph2d_pair_count(self.h, ctypes.byref(n)))
        return n.value

    def pair_list(self):
        """(off int64 [N+1], tri int32 [P]) on the device, input particle order."""
        P = self.pair_count()
        n = self._keep[0].shape[0]
        off = torch.empty(n + 1, dtype=torch.int64, device=self._dev())
        tri = torch.empty(max(P, 1), dtype=torch.int32, device=self._dev())
        req = ctypes.c_int64()
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_pair_list(self.h, _ptr(off), _ptr(tri), P, ctypes.byref(req)))
        return off, tri[:P]

    def stats(self) -> dict:
        s = Stats()
        check(self.lib, self.h, self.lib.sph2d_last_stats(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    # -- forward -----------------------------------------------------------------------
    def _alloc_out(self, n, moment_degree, mode, want_grad):
        dt = torch.float64 if _mode_id(mode) == 0 else torch.float32
        d = self._dev()
        g = torch.empty(n, dtype=dt, device=d)
        gr = torch.empty((n, 2), dtype=dt, device=d) if want_grad else None
        nm = num_moments(moment_degree)
        mo = torch.empty((n, nm), dtype=dt, device=d) if nm else None
        return g, gr, mo

    def boundary_integrals(self, particles, tris, kernel, H: float, moment_degree: int = -1,
                           mode="fp64", want_grad: bool = True):
        """Full path: cells, cull, closed-form pair integrals, per-particle sums."""
        src = particles.device
        p = as_particles(particles, self._dev())
        t = as_triangles(tris, self._dev())
        g, gr, mo = self._alloc_out(p.shape[0], moment_degree, mode, want_grad)
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_boundary_integrals(
            self.h, _ptr(p), p.shape[0], _ptr(t), t.shape[0], _kernel_id(kernel), float(H),
            int(moment_degree), _mode_id(mode), _ptr(g), _ptr(gr), _ptr(mo)))
        self._keep = (p, t)
        self._builds += 1
        if src.type != "cuda":
            g = g.to(src)
            gr = gr.to(src) if gr is not None else None
            mo = mo.to(src) if mo is not None else None
        return g, gr, mo

    def integrals_from_pairs(self, kernel, moment_degree: int = -1, mode="fp64", want_grad=True):
        n = self._keep[0].shape[0]
        g, gr, mo = self._alloc_out(n, moment_degree, mode, want_grad)
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_integrals_from_pairs(
            self.h, _kernel_id(kernel), int(moment_degree), _mode_id(mode), _ptr(g), _ptr(gr), _ptr(mo)))
        return g, gr, mo

    def pair_integrals(self, pairs, kernel, H: float, moment_degree: int = -1, mode="fp64"):
        """Independent pairs float64 [P, 8] -> [P, 3 + nm] (gamma, grad x, grad y, moments)."""
        q = pairs.to(device=self._dev(), dtype=torch.float64).contiguous()
        dt = torch.float64 if _mode_id(mode) == 0 else torch.float32
        out = torch.empty((q.shape[0], 3 + num_moments(moment_degree)), dtype=dt, device=self._dev())
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_pair_integrals(
            self.h, _ptr(q), q.shape[0], _kernel_id(kernel), float(H), int(moment_degree),
            _mode_id(mode), _ptr(out)))
        return out

    def field_integrals(self, vertex_values, kernel, mode="fp64", want_grad: bool = True, order: int = 1):
        """Lagrange fields over the pair list of the last build: node values [M, nodes, nf]
        (or [M, nodes]; nodes = 3, 6 or 10 for order 1, 2 or 3) -> value [N, nf], grad
        [N, nf, 2] (or None).  Order 1 is the piecewise-linear field."""
        vv = torch.as_tensor(vertex_values)
        if vv.dim() == 2:
            vv = vv[:, :, None]
        nf = vv.shape[2]
        if vv.shape[1] != (order + 1) * (order + 2) // 2:
            raise ValueError(f"order {order} needs {(order + 1) * (order + 2) // 2} node values per triangle")
        vv = vv.to(device=self._dev(), dtype=torch.float32).contiguous()
        n = self._keep[0].shape[0] if hasattr(self, "_keep") else 0
        dt = torch.float64 if _mode_id(mode) == 0 else torch.float32
        val = torch.empty((n, nf), dtype=dt, device=self._dev())
        gr = torch.empty((n, nf, 2), dtype=dt, device=self._dev()) if want_grad else None
        self._bind_stream()
        if order == 1:
            rc = self.lib.sph2d_field_integrals(
                self.h, _kernel_id(kernel), _mode_id(mode), _ptr(vv), int(nf), _ptr(val), _ptr(gr))
        else:
            rc = self.lib.sph2d_field_integrals_p(
                self.h, _kernel_id(kernel), _mode_id(mode), int(order), _ptr(vv), int(nf), _ptr(val), _ptr(gr))
        check(self.lib, self.h, rc)
        return val, gr

    # -- boundary pressure coupling (Appendix A) -----------------------------------------
    def mls_pressure(self, volume, pressure, points, kernel, mode="fp64"):
        """MLS pressure of the build's particles at points [Q, 2] -> [Q]."""
        vol = torch.as_tensor(volume).to(device=self._dev(), dtype=torch.float32).contiguous()
        pr = torch.as_tensor(pressure).to(device=self._dev(), dtype=torch.float32).contiguous()
        pts = torch.as_tensor(points).to(device=self._dev(), dtype=torch.float32).reshape(-1, 2).contiguous()
        dt = torch.float64 if _mode_id(mode) == 0 else torch.float32
        out = torch.empty(pts.shape[0], dtype=dt, device=self._dev())
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_mls_pressure(
            self.h, _kernel_id(kernel), _mode_id(mode), _ptr(vol), _ptr(pr), _ptr(pts), pts.shape[0], _ptr(out)))
        return out

    def boundary_pressure(self, density, pressure, volume, rho0_b: float, kernel, mode="fp64", model: int = 2):
        """Boundary pressure acceleration [N, 2] of the build's particles (model 1: vertex
        pressures, model 2: contact-point pressures)."""
        dev = self._dev()
        rho = torch.as_tensor(density).to(device=dev, dtype=torch.float32).contiguous()
        pr = torch.as_tensor(pressure).to(device=dev, dtype=torch.float32).contiguous()
        vol = torch.as_tensor(volume).to(device=dev, dtype=torch.float32).contiguous()
        n = self._keep[0].shape[0] if hasattr(self, "_keep") else 0
        dt = torch.float64 if _mode_id(mode) == 0 else torch.float32
        acc = torch.empty((n, 2), dtype=dt, device=dev)
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_boundary_pressure(
            self.h, _kernel_id(kernel), _mode_id(mode), int(model), _ptr(rho), _ptr(pr), _ptr(vol),
            float(rho0_b), _ptr(acc)))
        return acc

    # -- adjoint -----------------------------------------------------------------------
    def backward(self, particles, tris, kernel, H: float, d_gamma, mode="fp64", d_grad=None):
        """dL/dx [N, 2] and dL/dvertices [M, 6] from dL/dgamma [N] and optionally
        dL/dgrad gamma [N, 2]."""
        p = as_particles(particles, self._dev())
        t = as_triangles(tris, self._dev())
        dt = torch.float64 if _mode_id(mode) == 0 else torch.float32
        dg = d_gamma.to(device=self._dev(), dtype=dt).contiguous()
        dgr = d_grad.to(device=self._dev(), dtype=dt).contiguous() if d_grad is not None else None
        dp = torch.empty((p.shape[0], 2), dtype=dt, device=self._dev())
        dtr = torch.empty((t.shape[0], 6), dtype=dt, device=self._dev())
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_boundary_integrals_backward(
            self.h, _ptr(p), p.shape[0], _ptr(t), t.shape[0], _kernel_id(kernel), float(H),
            _mode_id(mode), _ptr(dg), _ptr(dgr) if dgr is not None else None, _ptr(dp), _ptr(dtr)))
        self._keep = (p, t)       # the rebuilt pair list points at these
        self._builds += 1
        return dp, dtr

    def backward_from_pairs(self, kernel, d_gamma, mode="fp64", d_grad=None):
        """As backward, over the pair list of the last build (no cull): dL/dx [N, 2] and
        dL/dvertices [M, 6] of that build's particles and triangles."""
        if getattr(self, "_keep", None) is None:
            raise _lib.Sph2dError(4, "no pair list built")
        n, m = self._keep[0].shape[0], self._keep[1].shape[0]
        dt = torch.float64 if _mode_id(mode) == 0 else torch.float32
        dg = d_gamma.to(device=self._dev(), dtype=dt).contiguous()
        dgr = d_grad.to(device=self._dev(), dtype=dt).contiguous() if d_grad is not None else None
        dp = torch.empty((n, 2), dtype=dt, device=self._dev())
        dtr = torch.empty((m, 6), dtype=dt, device=self._dev())
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_backward_from_pairs(
            self.h, _kernel_id(kernel), _mode_id(mode), _ptr(dg), _ptr(dgr) if dgr is not None else None,
            _ptr(dp), _ptr(dtr)))
        return dp, dtr

    # -- learned surrogate -------------------------------------------------------------
    def surrogate_init(self, kernel, seed: int = 0):
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_init(self.h, _kernel_id(kernel), int(seed)))
        return self

    def surrogate_train(self, pairs, H: float, epochs: int, batch: int = 4096, lr: float = 3e-3,
                        weight_decay: float = 0.0, seed: int = 0):
        """Train on independent pairs float64 [P, 8]; returns (last batch loss, pairs used)."""
        q = pairs.to(device=self._dev(), dtype=torch.float64).contiguous()
        loss = ctypes.c_double()
        used = ctypes.c_int64()
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_train(
            self.h, _ptr(q), q.shape[0], float(H), int(epochs), int(batch), float(lr),
            float(weight_decay), int(seed), ctypes.byref(loss), ctypes.byref(used)))
        return loss.value, used.value

    def surrogate_pairs(self, pairs, H: float):
        """Independent pairs float64 [P, 8] -> (float32 [P, 3] gamma and grad, int32 [P] accepted)."""
        q = pairs.to(device=self._dev(), dtype=torch.float64).contiguous()
        out = torch.empty((q.shape[0], 3), dtype=torch.float32, device=self._dev())
        acc = torch.empty(q.shape[0], dtype=torch.int32, device=self._dev())
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_pairs(self.h, _ptr(q), q.shape[0], float(H),
                                                                _ptr(out), _ptr(acc)))
        return out, acc

    def surrogate_forward(self, x):
        """Raw network on canonical inputs float32 [B, 6] -> float32 [B, 3]."""
        xx = x.to(device=self._dev(), dtype=torch.float32).contiguous()
        y = torch.empty((xx.shape[0], 3), dtype=torch.float32, device=self._dev())
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_forward(self.h, _ptr(xx), xx.shape[0], _ptr(y)))
        return y

    def surrogate_grad(self, x, t):
        """(parameter gradient float32 [SURROGATE_PARAMS], loss) of one batch."""
        xx = x.to(device=self._dev(), dtype=torch.float32).contiguous()
        tt = t.to(device=self._dev(), dtype=torch.float32).contiguous()
        g = torch.empty(_lib.SURROGATE_PARAMS, dtype=torch.float32, device=self._dev())
        loss = torch.empty(1, dtype=torch.float32, device=self._dev())
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_grad(self.h, _ptr(xx), _ptr(tt), xx.shape[0],
                                                               _ptr(g), _ptr(loss)))
        return g, loss

    def surrogate_params(self) -> torch.Tensor:
        p = torch.empty(_lib.SURROGATE_PARAMS, dtype=torch.float32)
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_get_params(self.h, _ptr(p), p.numel()))
        return p

    def set_surrogate_audit(self, period: int = 64, tol: float = 1e-3):
        """Serving audit: about 1 in `period` accepted pairs (0: off) judged by the analytic path;
        a call with an audited error above `tol` is evaluated analytically throughout."""
        check(self.lib, self.h, self.lib.sph2d_surrogate_set_audit(self.h, int(period), float(tol)))
        return self

    def set_surrogate_engine(self, engine: str = "mma_sync"):
        """Serving tensor-core engine: "mma_sync" (register-chained mma.sync) or "tcgen05"."""
        check(self.lib, self.h, self.lib.sph2d_surrogate_set_engine(self.h, {"mma_sync": 0, "tcgen05": 1}[engine]))
        return self

    def set_surrogate_train_engine(self, engine: str = "mma_sync"):
        """Tensor-core engine of the training GEMMs: "mma_sync" or "tcgen05"."""
        check(self.lib, self.h,
              self.lib.sph2d_surrogate_set_train_engine(self.h, {"mma_sync": 0, "tcgen05": 1}[engine]))
        return self

    def set_surrogate_params(self, p):
        q = torch.as_tensor(p, dtype=torch.float32).contiguous().cpu()
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_set_params(self.h, _ptr(q), q.numel()))

    def surrogate_save(self, path: str):
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_save(self.h, str(path).encode()))

    def surrogate_load(self, path: str):
        self._bind_stream()
        check(self.lib, self.h, self.lib.sph2d_surrogate_load(self.h, str(path).encode()))
        return self


def measure_fma_peak(device: int = 0, precision: str = "fp64", seconds: float = 0.2) -> float:
    """Measured FMA throughput (TFLOP/s) of one GPU in FP64 or FP32 (the library's microbenchmark)."""
    lib = _lib.load()
    out = ctypes.c_double()
    st = lib.sph2d_measure_fma_peak(int(device), 0 if precision == "fp64" else 1, float(seconds), ctypes.byref(out))
    if st != 0:
        raise _lib.Sph2dError(f"sph2d_measure_fma_peak: {_lib.STATUS.get(st, st)}")
    return float(out.value)


_contexts: dict[int, Context] = {}


def context(device: int | None = None) -> Context:
    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _contexts:
        _contexts[d] = Context(d)
    return _contexts[d]


def boundary_integrals(particles, tris, kernel, H: float, moment_degree: int = -1, mode="fp64",
                       want_grad: bool = True):
    """gamma [N], grad_gamma [N, 2] (or None), moments [N, nm] (or None)."""
    return context().boundary_integrals(particles, tris, kernel, H, moment_degree, mode, want_grad)


def pair_integrals(pairs, kernel, H: float, moment_degree: int = -1, mode="fp64"):
    return context().pair_integrals(pairs, kernel, H, moment_degree, mode)


class BoundaryGamma(torch.autograd.Function):
    """(gamma, grad gamma)(particles, triangles) with the library's adjoint kernels as backward.

    Gradients flow to particle positions (x, y) and triangle vertices through both outputs
    (the grad gamma path uses the second-order kernels)."""

    @staticmethod
    def forward(ctx, particles, tris, kernel, H, mode):
        c = context()
        g, gr, _ = c.boundary_integrals(particles, tris, kernel, H, -1, mode, True)
        ctx.save_for_backward(particles, tris)
        ctx.kernel, ctx.H, ctx.mode = kernel, H, mode
        ctx.build = c._builds
        return g, gr

    @staticmethod
    def backward(ctx, d_gamma, d_grad):
        particles, tris = ctx.saved_tensors
        if d_gamma is None:
            d_gamma = torch.zeros(particles.shape[0], dtype=particles.dtype, device=particles.device)
        c = context()
        if c._builds == ctx.build:
            # the context still holds this forward's pair list (saved tensors are checked for
            # in-place changes by autograd): no second cull
            dp, dt = c.backward_from_pairs(ctx.kernel, d_gamma, ctx.mode, d_grad)
        else:
            dp, dt = c.backward(particles, tris, ctx.kernel, ctx.H, d_gamma, ctx.mode, d_grad)
        gp = torch.zeros_like(particles)
        gp[:, :2] = dp.to(particles.dtype)
        return gp, dt.to(tris.dtype).reshape(tris.shape), None, None, None
