"""Synthetic reduced objects for the batched dictionary sweep.

Each object is given directly by reduced data of size r (shared basis for the
three directions): K_r Hermitian PSD with a log-uniform spectrum in
[1e-6, 1e2], C_r Hermitian PD with a log-uniform spectrum in [1e-3, 1],
b ~ CN(0, I) (r x 3), and the quantities the tensor and certificate formulas
need (c00 and the certificate Gram matrix G).

The Gram matrix is generated as if a random orthonormal basis U of a large
space (N = 4096) were given, together with components orthogonal to U:
Phi = [C o_1, C o_2, C o_3 | K U | C U] = U [B | K_r | C_r] + Y with
U^H Y = 0, so G = Phi^H Phi = [B|K_r|C_r]^H [B|K_r|C_r] + Y^H Y.  Only Y^H Y
enters G, so Y is drawn directly as a (2r+3) x (2r+3) matrix, which has the
same distribution as drawing it in the 4096 - r dimensional complement.
c00 = Re(B^H C_r^-1 B) + Z^T Z keeps the imaginary tensor part PSD.
K_r is split as K_out + K_in (both PSD, same eigenvectors) so that a
permeability scale s_mu can act as K_out + K_in / s_mu.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ReducedObject:
    r: int
    K_out: np.ndarray     # r x r complex128 Hermitian PSD
    K_in: np.ndarray      # r x r complex128 Hermitian PSD (mu_r-dependent part)
    C: np.ndarray         # r x r complex128 Hermitian PD
    B: np.ndarray         # r x 3 complex128
    c00: np.ndarray       # 3 x 3 float64
    G: np.ndarray         # (2r+3) x (2r+3) complex128 Hermitian PSD
    alpha: float = 1.0
    alpha_lb: float = 1.0 / np.sqrt(2.0)
    vol_B: float = 1.0

    @property
    def K(self) -> np.ndarray:
        return self.K_out + self.K_in


def _haar(rng, n):
    Z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R)
    return Q * (d / np.abs(d))[None, :]


def _herm(Q, lam):
    H = (Q * lam[None, :]) @ Q.conj().T
    return 0.5 * (H + H.conj().T)


def reduced_object(seed: int, index: int, r: int, *, k_range=(-6.0, 2.0), c_range=(-3.0, 0.0),
                   y_scale: float = 0.05) -> ReducedObject:
    """One synthetic reduced object of size r, seeded by (seed, index)."""
    rng = np.random.default_rng([seed, index])
    Q = _haar(rng, r)
    lam = 10.0 ** rng.uniform(*k_range, size=r)
    f = rng.uniform(0.0, 1.0, size=r)
    K_out = _herm(Q, lam * (1.0 - f))
    K_in = _herm(Q, lam * f)
    Qc = _haar(rng, r)
    C = _herm(Qc, 10.0 ** rng.uniform(*c_range, size=r))
    B = (rng.standard_normal((r, 3)) + 1j * rng.standard_normal((r, 3))) / np.sqrt(2.0)
    Z = rng.standard_normal((3, 3))
    CinvB = np.linalg.solve(C, B)
    c00 = np.real(B.conj().T @ CinvB)
    c00 = 0.5 * (c00 + c00.T) + Z.T @ Z
    PsiU = np.concatenate([B, K_out + K_in, C], axis=1)
    m = 2 * r + 3
    colnorm = np.linalg.norm(PsiU, axis=0)
    Y = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(2.0 * m)
    Y = Y * (y_scale * colnorm)[None, :]
    G = PsiU.conj().T @ PsiU + Y.conj().T @ Y
    G = 0.5 * (G + G.conj().T)
    return ReducedObject(r=r, K_out=K_out, K_in=K_in, C=C, B=B, c00=c00, G=G)


def reduced_dictionary(n_obj: int, seed: int = 20230711, r_lo: int = 8, r_hi: int = 96,
                       **kw) -> list:
    """n_obj objects with r drawn uniformly from {r_lo, ..., r_hi}."""
    rng = np.random.default_rng(seed)
    rs = rng.integers(r_lo, r_hi + 1, size=n_obj)
    return [reduced_object(seed, i, int(rs[i]), **kw) for i in range(n_obj)]
