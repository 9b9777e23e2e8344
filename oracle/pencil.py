"""Second, independent reduced sweep through the Hermitian pencil (K_r + eps M_r, C_r).

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.

For one basis shared by the three directions, the generalized eigenproblem
(K_r + eps M_r) v = lambda C_r v with V^H C_r V = I gives
A(omega)^-1 = V (Lambda - i omega I)^-1 V^H, so
p_i(omega) = i omega V (Lambda - i omega I)^-1 V^H b_i
without any LU factorisation.  Used only to pin ``rom.reduced_solve``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pencil_solve(model, omegas) -> list:
    """p_i^M[omega] for a shared-basis ReducedModel; list of three (n_w, r) arrays."""
    w = np.asarray(omegas, dtype=np.float64)
    A0 = model.K[0][0] + model.Me[0]
    A0 = 0.5 * (A0 + A0.conj().T)
    C = 0.5 * (model.C[0][0] + model.C[0][0].conj().T)
    lam, V = sla.eigh(A0, C)
    out = []
    for i in range(3):
        c = V.conj().T @ model.b(i)
        z = c[None, :] / (lam[None, :] - 1j * w[:, None])
        out.append((1j * w)[:, None] * (z @ V.T))
    return out
