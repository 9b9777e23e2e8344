"""Snapshot SVD and truncation (Sect. 4.1, Eqs. (13)-(15)).

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.
"""
from __future__ import annotations

import numpy as np


def truncation_rank(s: np.ndarray, tol_sigma: float, r_max: int | None = None) -> int:
    """Number of retained modes: every s_n with s_n / s_1 >= TOL_Sigma, capped at r_max.

    The printed rule below Eq. (15) is garbled (it states s_M / s_1 < TOL);
    the reading taken is that the retained singular values are those not
    below TOL_Sigma relative to the largest one.  TOL_Sigma = 0 keeps all.
    """
    if s.size == 0 or s[0] == 0.0:
        return 0
    r = int(np.count_nonzero(s / s[0] >= tol_sigma))
    if r_max is not None:
        r = min(r, int(r_max))
    return r


def truncated_svd(D: np.ndarray, tol_sigma: float, r_max: int | None = None):
    """U^M, Sigma^M, (V^M)^H of Eq. (15) for one snapshot matrix D (N x N_s).

    Uses LAPACK's SVD (numpy.linalg.svd) on D itself, Eq. (14), then keeps
    the leading M columns.
    """
    U, s, Vh = np.linalg.svd(D, full_matrices=False)
    r = truncation_rank(s, tol_sigma, r_max)
    return U[:, :r], s[:r], Vh[:r], s
