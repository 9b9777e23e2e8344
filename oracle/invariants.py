"""Rotation-invariant features of the MPT spectral signature (Sect. 1).

Under a rotation of the object, each 3 x 3 coefficient matrix transforms as
M' = Q M Q^T, so the eigenvalues of the real symmetric parts R~ = N0 + R and I
at each frequency do not depend on the object's orientation; dictionary
matching compares those eigenvalues.

Test infrastructure only: imported by tests/, never by the product path.
"""
from __future__ import annotations

import numpy as np


def mpt_invariants(M: np.ndarray) -> np.ndarray:
    """Eigenvalues (ascending) of each symmetric 3 x 3 matrix of M (..., 3, 3).

    The symmetric part 0.5 (M + M^T) is used (R~ and I are symmetric up to
    rounding); numpy.linalg.eigvalsh (LAPACK) does the decomposition.
    """
    M = np.asarray(M, dtype=np.float64)
    S = 0.5 * (M + np.swapaxes(M, -1, -2))
    return np.linalg.eigvalsh(S)
