"""ctypes binding to libsph2d.so (include/sph2d.h).  Argument marshalling only.

The library must be built first (``paper_2507_21686_gb300.build.build()`` or
``__graft_entry__.build()``); loading fails loudly otherwise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB

SPH2D_OK = 0
STATUS = {
    0: "SPH2D_OK",
    1: "SPH2D_ERR_INVALID_ARG",
    2: "SPH2D_ERR_NONFINITE_INPUT",
    3: "SPH2D_ERR_CAPACITY",
    4: "SPH2D_ERR_NOT_BUILT",
    5: "SPH2D_ERR_CUDA",
    6: "SPH2D_ERR_UNSUPPORTED",
    7: "SPH2D_ERR_OUT_OF_MEMORY",
}
KERNELS = {"wendland_c2": 0, "wendland_c4": 1, "wendland_c6": 2, "cubic_spline": 3}
MODES = {"fp64": 0, "fp32_fixup": 1, "surrogate": 2, "fp32_hybrid": 3}

# every symbol the header declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
_ST = ctypes.c_int


class Stats(ctypes.Structure):
    _fields_ = [("n_particles", ctypes.c_int64), ("n_triangles", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("n_fixup", ctypes.c_int64),
                ("n_fallback", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("n_candidates", ctypes.c_int64),
                ("n_launches", ctypes.c_int64),
                ("n_audit", ctypes.c_int64), ("n_audit_over", ctypes.c_int64),
                ("audit_max_err", ctypes.c_double), ("n_redo", ctypes.c_int64),
                ("n_mma_timeouts", ctypes.c_int64)]


SIGNATURES = {
    "sph2d_version": (_I, []),
    "sph2d_init": (_ST, [ctypes.POINTER(_P), _I, _P]),
    "sph2d_destroy": (_ST, [_P]),
    "sph2d_set_stream": (_ST, [_P, _P]),
    "sph2d_last_error": (ctypes.c_char_p, [_P]),
    "sph2d_last_stats": (_ST, [_P, ctypes.POINTER(Stats)]),
    "sph2d_build_cells": (_ST, [_P, _P, _I64, _P, _I64, _D]),
    "sph2d_pair_count": (_ST, [_P, ctypes.POINTER(_I64)]),
    "sph2d_pair_list": (_ST, [_P, _P, _P, _I64, ctypes.POINTER(_I64)]),
    "sph2d_boundary_integrals": (_ST, [_P, _P, _I64, _P, _I64, _I, _D, _I, _I, _P, _P, _P]),
    "sph2d_integrals_from_pairs": (_ST, [_P, _I, _I, _I, _P, _P, _P]),
    "sph2d_pair_integrals": (_ST, [_P, _P, _I64, _I, _D, _I, _I, _P]),
    "sph2d_boundary_integrals_backward": (_ST, [_P, _P, _I64, _P, _I64, _I, _D, _I, _P, _P, _P, _P]),
    "sph2d_backward_from_pairs": (_ST, [_P, _I, _I, _P, _P, _P, _P]),
    "sph2d_pair_list_integrals_noalloc": (_ST, [_P, _I64, _P, _I64, _P, _P, _I64, _I, _D, _I, _P, _P, _P]),
    "sph2d_field_integrals": (_ST, [_P, _I, _I, _P, _I, _P, _P]),
    "sph2d_field_integrals_p": (_ST, [_P, _I, _I, _I, _P, _I, _P, _P]),
    "sph2d_mls_pressure": (_ST, [_P, _I, _I, _P, _P, _P, _I64, _P]),
    "sph2d_boundary_pressure": (_ST, [_P, _I, _I, _I, _P, _P, _P, _D, _P]),
    "sph2d_surrogate_init": (_ST, [_P, _I, ctypes.c_uint64]),
    "sph2d_surrogate_train": (_ST, [_P, _P, _I64, _D, _I, _I, _D, _D, ctypes.c_uint64,
                                    ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "sph2d_surrogate_pairs": (_ST, [_P, _P, _I64, _D, _P, _P]),
    "sph2d_surrogate_forward": (_ST, [_P, _P, _I64, _P]),
    "sph2d_surrogate_grad": (_ST, [_P, _P, _P, _I64, _P, _P]),
    "sph2d_surrogate_get_params": (_ST, [_P, _P, _I64]),
    "sph2d_surrogate_set_params": (_ST, [_P, _P, _I64]),
    "sph2d_surrogate_set_audit": (_ST, [_P, _I, _D]),
    "sph2d_surrogate_set_engine": (_ST, [_P, _I]),
    "sph2d_surrogate_set_train_engine": (_ST, [_P, _I]),
    "sph2d_measure_fma_peak": (_ST, [_I, _I, _D, ctypes.POINTER(ctypes.c_double)]),
    "sph2d_surrogate_save": (_ST, [_P, ctypes.c_char_p]),
    "sph2d_surrogate_load": (_ST, [_P, ctypes.c_char_p]),
}

SURROGATE_PARAMS = 8963

_lib = None


class Sph2dError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB) -> ctypes.CDLL:
    """Load libsph2d and bind every declared symbol (raises if any is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsph2d not built ({path} missing): run paper_2507_21686_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(lib, ctx, status: int) -> None:
    if status != SPH2D_OK:
        msg = lib.sph2d_last_error(ctx)
        raise Sph2dError(status, msg.decode() if msg else "")
