"""Roofline inputs: algorithmic operation counts of the pair formula and the ALU peaks.

The op counts come from ``libsph2d_opcount.so``, which instantiates the same closed-form
pair code as the CUDA kernels with an operation-counting scalar type (add, mul, div, sqrt and
each transcendental = 1 flop, fma = 2).  Three counts per pair:
    "method"  the closed form in plain arithmetic: the algorithmic work of the roofline
    "fp32"    the compensated FP32 form (error-free transformations counted as work)
    "fp64"    the FP64 path as it runs
Peaks are derived from GB300 unit counts and clocks.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .build import OPCOUNT_LIB

KERNELS = {"wendland_c2": 0, "wendland_c4": 1, "wendland_c6": 2, "cubic_spline": 3}

# GB300: 152 SMs; per SM and clock: 128 FP32 lanes (FMA = 2 flops).  Max SM clock 2070 MHz.
SMS = 152
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(mhz: float = SM_MAX_MHZ) -> float:
    """FMA-flop peak (every lane issuing one FMA per clock)."""
    return SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def fp32_lane_op_peak_tops(mhz: float = SM_MAX_MHZ) -> float:
    """FP32 lane-operation peak: every FP32 lane issuing one add, mul or fma per clock."""
    return SMS * FP32_LANES_PER_SM * mhz * 1e6 / 1e12


# NVIDIA's published dense FP64 rate for the GB300 (Blackwell Ultra) GPU, at boost clock
FP64_PEAK_TFLOPS_NOMINAL = 1.25

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(OPCOUNT_LIB)
        _lib.sph2d_count_pair_ops.restype = ctypes.c_int64
        _lib.sph2d_count_pair_ops.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_void_p, ctypes.c_void_p]
    return _lib


def _degree(moments) -> int:
    """moments: True (all ten, degree 3), False (none) or a moment degree -1..3."""
    if isinstance(moments, bool):
        return 3 if moments else -1
    return int(moments)


COUNT_KINDS = {"fp64": 0, "fp32": 1, "method": 2}


def _kind(kind) -> int:
    """'fp64' | 'fp32' | 'method' (True / False: the compensated FP32 form / the FP64 path)."""
    if isinstance(kind, bool):
        return 1 if kind else 0
    return COUNT_KINDS[kind]


def pair_ops(kernel, moments, kind, local_tri) -> tuple[int, np.ndarray]:
    """(flops, [add, mul, fma, div, sqrt, transcendental, other]) for one local-frame pair."""
    lib = _load()
    l = np.ascontiguousarray(local_tri, dtype=np.float64).reshape(6)
    out = np.zeros(7, dtype=np.int64)
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    f = lib.sph2d_count_pair_ops(k, _degree(moments), _kind(kind), l.ctypes.data, out.ctypes.data)
    return int(f), out


def mean_flops_per_pair(kernel, moments, kind, local_tris: np.ndarray) -> float:
    """Average over a sample of real pairs (rows of local-frame triangles, H = 1)."""
    return float(np.mean([pair_ops(kernel, moments, kind, t)[0] for t in local_tris]))


def mean_ops_per_pair(kernel, moments, kind, local_tris: np.ndarray) -> float:
    """Floating-point operations per pair with fma counted once (lane-operations)."""
    return float(np.mean([pair_ops(kernel, moments, kind, t)[1][:6].sum() for t in local_tris]))
