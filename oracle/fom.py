"""Full-order solutions and the Full Matrix Method (FMM), Sect. 3.1-3.2.

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.

Notation: q_i[omega] are the full-order solution coefficients of direction i
(Eq. (9)), o~_i the theta~^(0) coefficients, x_i the coefficients of
e_i x xi, and alpha the object size.  With one discrete space for theta~^(0)
and theta^(1) (Remark 3.1): C^(1) = C^(2) = C, s_i = t_i = C x_i and
c_ij = x_i^T C x_j.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def system_matrix(problem, omega: float):
    """A[omega] = K - i omega C + eps M (Sect. 3.1, below Eq. (9))."""
    N = problem.N
    return (sp.csc_matrix(problem.K, dtype=np.complex128)
            + sp.diags(problem.eps * problem.M - 1j * omega * problem.C, format="csc",
                       shape=(N, N)))


def source(problem, omega: float) -> np.ndarray:
    """r(theta_i^(0)) = i omega C (o~_i + x_i) for i = 1..3, as an N x 3 array.

    The right-hand side of Eq. (7a) is i nu theta_i^(0) in B; its weak form is
    i omega c(theta_i^(0), w), so the load vector is i omega C times the total
    theta^(0) coefficients.
    """
    o_total = problem.o_tilde + problem.x
    return (1j * omega) * (problem.C[:, None] * o_total.T)


def full_order_solution(problem, omega: float) -> np.ndarray:
    """Solve Eq. (9) for q_i[omega], i = 1..3, by sparse LU; returns N x 3."""
    lu = spla.splu(system_matrix(problem, omega))
    return lu.solve(source(problem, omega))


def fmm_R(problem, q: np.ndarray) -> np.ndarray:
    """Eq. (11): R_ij = -alpha^3/4 conj(q_i)^T K q_j, real part taken.

    R is a real symmetric tensor (Eq. (6b)); the discrete quadratic form can
    carry a rounding-level imaginary part for i != j, which is dropped.
    """
    a3 = problem.alpha ** 3
    H = q.conj().T @ (problem.K @ q)
    return -a3 / 4.0 * H.real


def fmm_I(problem, q: np.ndarray, omega: float) -> np.ndarray:
    """Eq. (12) term by term, with C^(1) = C^(2) = C and s = t = C x (Remark 3.1)."""
    a3 = problem.alpha ** 3
    C = problem.C
    o = problem.o_tilde            # 3 x N, theta~^(0) coefficients
    x = problem.x                  # 3 x N, e_i x xi coefficients
    s = C[None, :] * x             # s_i = t_i = C x_i
    oCo = o @ (C[:, None] * o.T)   # o_i^T C^(1) o_j
    c = x @ (C[:, None] * x.T)     # c_ij
    so = s @ o.T                   # (s_i^T o_j)
    qCq = q.conj().T @ (C[:, None] * q)          # conj(q_i)^T C q_j
    oCq = o @ (C[:, None] * q)                   # o_i^T C^(2) q_j
    oCqbar = (o @ (C[:, None] * q.conj())).T     # [i,j] = o_j^T C^(2) conj(q_i)
    tq = s @ q                                   # t_i^T q_j
    tqbar = (s @ q.conj()).T                     # [i,j] = t_j^T conj(q_i)
    inner = oCo + c + so + so.T + np.real(qCq + oCq + oCqbar + tq + tqbar)
    return omega * a3 / 4.0 * inner


def fmm_signature(problem, omegas):
    """R[omega], I[omega] (n_w x 3 x 3 each) by full-order solves at every omega."""
    omegas = np.asarray(omegas, dtype=np.float64)
    R = np.empty((omegas.size, 3, 3))
    I = np.empty((omegas.size, 3, 3))
    for n, w in enumerate(omegas):
        q = full_order_solution(problem, w)
        R[n] = fmm_R(problem, q)
        I[n] = fmm_I(problem, q, w)
    return R, I
