"""sph2d: analytic 2-D SPH boundary integrals (arXiv 2507.21686) on GB300 (sm_103a).

Import is light: the CUDA library is loaded on first use of the API.
"""
__version__ = "1.0.0"

__all__ = ["boundary_integrals", "pair_integrals", "Context", "BoundaryGamma", "context",
           "KERNELS", "MODES"]

KERNELS = {"wendland_c2": 0, "wendland_c4": 1, "wendland_c6": 2, "cubic_spline": 3}
MODES = {"fp64": 0, "fp32_fixup": 1, "surrogate": 2}


def __getattr__(name):
    if name in ("boundary_integrals", "pair_integrals", "Context", "BoundaryGamma", "context"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
