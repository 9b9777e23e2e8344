"""Galerkin reduced-order model and the Matrix Method (Sects. 4.2-4.3).

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.

A ReducedModel holds, for the three directions i = 1..3 with (possibly
different) bases U_i, the omega-independent quantities the Matrix Method
precomputes (Eqs. (17)-(19)):

  K_ij = U_i^H K U_j,  C_ij = U_i^H C U_j,  Me_i = U_i^H (eps M) U_i,
  oCU_ij = o_i^T C U_j   (the o_i^T C_j^(2),M and t_i^M terms of Eq. (19)
                          added together, o_i = o~_i + x_i; Remark 3.1),
  c00_ij = o~_i^T C o~_j + c_ij + s_i^T o~_j + s_j^T o~_i.

The reduced source of direction i is U_i^H r_i = i omega (oCU_ii)^H.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ReducedModel:
    r: tuple                 # (r_1, r_2, r_3)
    K: list                  # 3 x 3 nested list of blocks K_ij (r_i x r_j)
    C: list                  # 3 x 3 nested list of blocks C_ij
    Me: list                 # 3 blocks U_i^H (eps M) U_i
    oCU: list                # 3 x 3 nested list of row vectors o_i^T C U_j (length r_j)
    c00: np.ndarray          # 3 x 3
    alpha: float = 1.0
    # certificate data (Lemma 4.2): Gram of Phi = [C o_1 C o_2 C o_3 | (K+eps M)U_d | C U_d ...]
    gram: np.ndarray | None = None
    gram_idx: list = field(default_factory=list)   # per direction: (src col, K-block slice, C-block slice)
    alpha_lb: float = 1.0 / np.sqrt(2.0)
    vol_B: float = 1.0
    eps_in_R: bool = False

    def b(self, i: int) -> np.ndarray:
        """b_i with U_i^H r_i = i omega b_i, i.e. b_i = U_i^H C o_i."""
        return self.oCU[i][i].conj()


def project(problem, U, *, eps_in_R: bool = False) -> ReducedModel:
    """Galerkin projection of the full-order matrices onto the POD bases (Eq. (17)).

    U is either one N x r basis shared by the three directions or a list of
    three bases.  K is applied as a sparse product; C and M are diagonal.
    """
    Us = list(U) if isinstance(U, (list, tuple)) else [U, U, U]
    Kd = problem.K
    Cd = problem.C
    KU = [Kd @ Ui for Ui in Us]
    CU = [Cd[:, None] * Ui for Ui in Us]
    K = [[Us[i].conj().T @ KU[j] for j in range(3)] for i in range(3)]
    Cb = [[Us[i].conj().T @ CU[j] for j in range(3)] for i in range(3)]
    if eps_in_R:
        K = [[K[i][j] + (problem.eps * (Us[i].conj().T @ (problem.M[:, None] * Us[j])))
              for j in range(3)] for i in range(3)]
        Me = [np.zeros((Ui.shape[1],) * 2, dtype=np.complex128) for Ui in Us]
    else:
        Me = [problem.eps * (Ui.conj().T @ (problem.M[:, None] * Ui)) for Ui in Us]
    o = problem.o_tilde + problem.x
    oCU = [[(o[i] * Cd) @ Us[j] for j in range(3)] for i in range(3)]
    ot, x = problem.o_tilde, problem.x
    s = Cd[None, :] * x
    so = s @ ot.T
    c00 = ot @ (Cd[:, None] * ot.T) + x @ (Cd[:, None] * x.T) + so + so.T
    return ReducedModel(r=tuple(Ui.shape[1] for Ui in Us), K=K, C=Cb, Me=Me, oCU=oCU, c00=c00,
                        alpha=problem.alpha, vol_B=problem.vol_B, eps_in_R=eps_in_R)


def from_reduced_object(obj, *, s_mu: float = 1.0) -> ReducedModel:
    """ReducedModel of a synthetic dictionary object (one basis for all directions).

    The permeability scale acts on the stiffness as K_out + K_in / s_mu; b,
    c00 and the Gram matrix are those of s_mu = 1.
    """
    K = obj.K_out + obj.K_in / s_mu
    r = obj.r
    Kb = [[K] * 3 for _ in range(3)]
    Cb = [[obj.C] * 3 for _ in range(3)]
    oCU = [[obj.B[:, i].conj()] * 3 for i in range(3)]
    idx = [(i, slice(3, 3 + r), slice(3 + r, 3 + 2 * r)) for i in range(3)]
    return ReducedModel(r=(r, r, r), K=Kb, C=Cb, Me=[np.zeros((r, r), complex)] * 3, oCU=oCU,
                        c00=obj.c00.copy(), alpha=obj.alpha, gram=obj.G, gram_idx=idx,
                        alpha_lb=obj.alpha_lb, vol_B=obj.vol_B)


def reduced_solve(model: ReducedModel, omegas) -> list:
    """p_i^M[omega] from Eq. (17): (K_ii + eps M_ii - i omega C_ii) p_i = i omega b_i.

    Returns a list of three arrays of shape (n_w, r_i), one dense LAPACK solve
    (numpy.linalg.solve, partial pivoting) per frequency and direction.
    """
    w = np.asarray(omegas, dtype=np.float64)
    out = []
    for i in range(3):
        A0 = model.K[i][i] + model.Me[i]
        A = A0[None, :, :] - 1j * w[:, None, None] * model.C[i][i][None, :, :]
        rhs = (1j * w)[:, None] * model.b(i)[None, :]
        out.append(np.linalg.solve(A, rhs[:, :, None])[:, :, 0])
    return out


def mm_tensors(model: ReducedModel, omegas, P: list):
    """Eq. (18) and Eq. (19) for every frequency; returns R, I of shape (n_w, 3, 3).

    R_ij = -alpha^3/4 Re(conj(p_i)^T K_ij p_j)   (real part: R is real, Eq. (6b));
    I_ij = omega alpha^3/4 (c00_ij + Re(conj(p_i)^T C_ij p_j + oCU_ij p_j
                                        + conj(oCU_ji p_i))).
    """
    w = np.asarray(omegas, dtype=np.float64)
    a3 = model.alpha ** 3
    R = np.empty((w.size, 3, 3))
    I = np.empty((w.size, 3, 3))
    for i in range(3):
        for j in range(3):
            Kp = P[j] @ model.K[i][j].T          # rows: (K_ij p_j)^T per omega
            Cp = P[j] @ model.C[i][j].T
            hK = np.einsum("wa,wa->w", P[i].conj(), Kp)
            hC = np.einsum("wa,wa->w", P[i].conj(), Cp)
            src = P[j] @ model.oCU[i][j] + np.conj(P[i] @ model.oCU[j][i])
            R[:, i, j] = -a3 / 4.0 * hK.real
            I[:, i, j] = w * a3 / 4.0 * (model.c00[i, j] + np.real(hC + src))
    return R, I


def rom_signature(model: ReducedModel, omegas):
    """On-line stage of Algorithm 1: R^PODP, I^PODP at every output frequency."""
    P = reduced_solve(model, omegas)
    R, I = mm_tensors(model, omegas, P)
    return R, I, P
