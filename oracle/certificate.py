"""A-posteriori error certificate, Lemma 4.2 (Eq. (20)).

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.

The residual of direction i for the PODP solution q_i = U_i p_i is
rho_i = r_i - A U_i p_i = i omega C o_i - (K + eps M) U_i p_i + i omega C U_i p_i
      = Phi_i w^(i),   Phi_i = [C o_i | (K + eps M) U_i | C U_i],
                       w^(i) = [i omega ; -p_i ; i omega p_i].
Its Riesz representer in the discrete space with inner-product matrix X has
norm ||r^_i||^2 = rho_i^H X^-1 rho_i = w^(i)H G^(ii) w^(i), with
G^(ij) = Phi_i^H X^-1 Phi_j.  The paper defers the definitions of w, G, the
norm and alpha_LB to its reference [Wilson & Ledger 2021]; the reading taken
here is X = K + eps M + omega_min C (real SPD), for which
|a(v, v)| >= ||v||_X^2 / sqrt(2) for all omega >= omega_min, so
alpha_LB = 1/sqrt(2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def inner_product_matrix(problem, omega_min: float):
    """X = K + eps M + omega_min C (sparse, real SPD)."""
    return (problem.K + sp.diags(problem.eps * problem.M + omega_min * problem.C)).tocsc()


def attach_gram(model, problem, U, X) -> None:
    """Form G = Phi^H X^-1 Phi for Phi = [C o_1, C o_2, C o_3 | (K+eps M)U_1 | C U_1 | ...].

    One sparse LU of X, applied to all columns of Phi.  For a shared basis the
    (K+eps M)U and C U blocks appear once.
    """
    Us = list(U) if isinstance(U, (list, tuple)) else [U]
    o = problem.o_tilde + problem.x
    cols = [problem.C * o[i] for i in range(3)]
    idx_blocks = []
    pos = 3
    for Ud in Us:
        r = Ud.shape[1]
        cols.extend(list(((problem.K @ Ud) + (problem.eps * problem.M)[:, None] * Ud).T))
        cols.extend(list((problem.C[:, None] * Ud).T))
        idx_blocks.append((slice(pos, pos + r), slice(pos + r, pos + 2 * r)))
        pos += 2 * r
    Phi = np.stack(cols, axis=1).astype(np.complex128)
    lu = spla.splu(sp.csc_matrix(X, dtype=np.float64))
    XiPhi = lu.solve(Phi.real) + 1j * lu.solve(Phi.imag)
    G = Phi.conj().T @ XiPhi
    model.gram = 0.5 * (G + G.conj().T)
    if len(Us) == 1:
        model.gram_idx = [(i, idx_blocks[0][0], idx_blocks[0][1]) for i in range(3)]
    else:
        model.gram_idx = [(i, idx_blocks[i][0], idx_blocks[i][1]) for i in range(3)]


def residual_weights(model, omega: float, p: list) -> list:
    """w^(i) placed in the columns of the stacked Gram matrix (one vector per direction)."""
    n = model.gram.shape[0]
    out = []
    for i in range(3):
        src, ks, cs = model.gram_idx[i]
        w = np.zeros(n, dtype=np.complex128)
        w[src] = 1j * omega
        w[ks] += -p[i]
        w[cs] += 1j * omega * p[i]
        out.append(w)
    return out


def certificate(model, omegas, P: list) -> np.ndarray:
    """(Delta[omega])_ij of Lemma 4.2 for every frequency; shape (n_w, 3, 3).

    ||r^_i||^2 = w^(i)H G w^(i), ||r^_i - r^_j||^2 = ||r^_i||^2 + ||r^_j||^2
    - 2 Re(w^(i)H G w^(j)), and
    Delta_ij = alpha^3 / (8 alpha_LB) (||r^_i||^2 + ||r^_j||^2 + ||r^_i - r^_j||^2).
    """
    w_all = np.asarray(omegas, dtype=np.float64)
    a3 = model.alpha ** 3
    out = np.empty((w_all.size, 3, 3))
    G = model.gram
    for n, w in enumerate(w_all):
        W = residual_weights(model, w, [P[i][n] for i in range(3)])
        GW = [G @ W[j] for j in range(3)]
        nrm = np.array([np.real(np.vdot(W[i], GW[i])) for i in range(3)])
        for i in range(3):
            for j in range(3):
                cross = np.real(np.vdot(W[i], GW[j]))
                diff = nrm[i] + nrm[j] - 2.0 * cross
                out[n, i, j] = a3 / (8.0 * model.alpha_lb) * (nrm[i] + nrm[j] + diff)
    return out


def residual_norms_direct(problem, U, omega: float, p: list, X) -> np.ndarray:
    """||r^_i||^2 computed from the full-order residual vector (pin for the Gram form)."""
    Us = list(U) if isinstance(U, (list, tuple)) else [U, U, U]
    o = problem.o_tilde + problem.x
    A = (sp.csc_matrix(problem.K, dtype=np.complex128)
         + sp.diags(problem.eps * problem.M - 1j * omega * problem.C))
    lu = spla.splu(sp.csc_matrix(X, dtype=np.float64))
    out = np.empty(3)
    for i in range(3):
        rho = 1j * omega * problem.C * o[i] - A @ (Us[i] @ p[i])
        z = lu.solve(rho.real) + 1j * lu.solve(rho.imag)
        out[i] = np.real(np.vdot(rho, z))
    return out


def residual_differences_direct(problem, U, omega: float, p: list, X) -> np.ndarray:
    """||r^_i - r^_j||^2 for every pair (i, j), from the explicit full-order residual vectors
    rho_i = i omega C o_i - A U_i p_i and one sparse LU of X: (rho_i - rho_j)^H X^-1 (rho_i - rho_j).
    Pin for the off-diagonal entries of Lemma 4.2, which the Gram form gets from a cross term."""
    Us = list(U) if isinstance(U, (list, tuple)) else [U, U, U]
    o = problem.o_tilde + problem.x
    A = (sp.csc_matrix(problem.K, dtype=np.complex128)
         + sp.diags(problem.eps * problem.M - 1j * omega * problem.C))
    lu = spla.splu(sp.csc_matrix(X, dtype=np.float64))
    rho = [1j * omega * problem.C * o[i] - A @ (Us[i] @ p[i]) for i in range(3)]
    out = np.empty((3, 3))
    for i in range(3):
        for j in range(3):
            d = rho[i] - rho[j]
            z = lu.solve(d.real) + 1j * lu.solve(d.imag)
            out[i, j] = np.real(np.vdot(d, z))
    return out
