"""Frequency grids: logarithmically spaced, both end points included."""
import numpy as np


def log_omegas(w_min: float, w_max: float, n: int) -> np.ndarray:
    """n angular frequencies log-spaced over [w_min, w_max] rad/s (inclusive)."""
    if n == 1:
        return np.array([float(w_min)])
    return np.logspace(np.log10(w_min), np.log10(w_max), n)
