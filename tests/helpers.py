"""Shared test infrastructure.  The error metrics and tolerances live in the package's
accuracy module (bench.py uses the same ones); this module re-exports them and adds the
oracle's per-pair row layout."""
from __future__ import annotations

import numpy as np

from paper_2507_21686_gb300.accuracy import (KERNEL_NAMES, MOMENT_ORDER, PAIR_FLOOR, TOL_FP32,  # noqa: F401
                                             TOL_FP64, TOL_SURROGATE, pair_rel_err, radial_moment, rel_err,
                                             scales)


def oracle_per_pair(o16: np.ndarray, nm: int) -> np.ndarray:
    """Oracle [P, 16] rows -> (gamma, gx, gy, M...) in the GPU per-pair layout."""
    return np.concatenate([o16[:, 0:3], o16[:, 5:5 + nm]], axis=1)
