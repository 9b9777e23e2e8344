"""Snapshot matrices D_i (Sect. 4.1, Eq. (13)).

``full_order_snapshots`` solves the full-order system of Eq. (9),
A[omega] q_i = i omega C o_i, at each snapshot frequency with a sparse direct
factorisation; this is the paper's off-line data generation, outside the
reduced-order path.  ``synthetic_snapshot_matrix`` makes large snapshot
matrices with a prescribed singular-value decay for grids where a sparse
direct solve is out of reach (the N = 2.6M and 6.2M grids).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .fit import FitProblem


def full_order_snapshots(problem: FitProblem, omegas) -> np.ndarray:
    """D with shape (3, N, N_s): D[i][:, n] = q_i[omega_n] (complex128)."""
    omegas = np.asarray(omegas, dtype=np.float64)
    D = np.empty((3, problem.N, omegas.size), dtype=np.complex128)
    for n, w in enumerate(omegas):
        lu = spla.splu(problem.A(w))
        D[:, :, n] = lu.solve(problem.rhs(w)).T
    return D


def synthetic_snapshot_matrix(N: int, n_s: int, seed: int, *, decay: float = 0.55,
                              n_dirs: int = 3, dtype=np.complex128) -> np.ndarray:
    """Random (n_dirs, N, n_s) snapshot stack with geometric singular-value decay.

    Column n of direction i is Z_i t_n where Z_i has i.i.d. CN(0,1)/sqrt(N)
    entries and T_i = diag(decay^k) V_i^H with V_i Haar-unitary, so the
    singular values are close to decay^k (k = 0..n_s-1).
    """
    rng = np.random.default_rng(seed)
    out = np.empty((n_dirs, N, n_s), dtype=dtype)
    s = decay ** np.arange(n_s)
    for i in range(n_dirs):
        V = _haar(rng, n_s)
        T = (s[:, None] * V.conj().T).astype(np.complex128)
        for c0 in range(0, N, 1 << 20):
            c1 = min(N, c0 + (1 << 20))
            Z = (rng.standard_normal((c1 - c0, n_s)) + 1j * rng.standard_normal((c1 - c0, n_s)))
            Z *= 1.0 / np.sqrt(2.0 * N)
            out[i, c0:c1] = (Z @ T).astype(dtype)
    return out


def _haar(rng, n):
    Z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R)
    return Q * (d / np.abs(d))[None, :]
