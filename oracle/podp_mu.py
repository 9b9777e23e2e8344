"""PODP in the relative permeability: the Matrix Method with mu_r as a second parameter.

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.

Sect. 4.2 notes that the precomputation behind Eqs. (17)-(19) carries over to
parameters other than omega.  This module takes the parameter s that scales
mu_r in every cell of the object B (mu_r -> s mu_r).  Readings, where the
paper gives no formulas:

* K is linear in mu_r^-1 cell by cell (Eq. (10a)), so
  K(s) = K_out + K_in / s with K_in the part carried by the cells of B;
  C and M do not depend on mu_r.
* theta~^(0) depends on mu_r (Eq. (5) with mu_r in the curl-curl term): its
  coefficients solve (K(s) + eps_s M_Omega) o~(s) = -K(s) x, a second full-order
  problem.  It is reduced the same way as theta^(1): a POD basis V of static
  snapshots o~(s_l) (one truncated SVD, Sect. 4.1), and its Galerkin system
  (V^H K(s) V + V^H eps_s M_Omega V) y = -V^H K(s) x for y (m x 3), o~ ~= V y.
  Every reduced operator is affine in 1/s.
* With o(s) = x + V y(s), the quantities of Eqs. (17)-(19) that depend on
  theta^(0) become b(s) = U^H C o(s), c00(s) = o(s)^T C o(s) and
  N0(s) = alpha^3 (|B| - (1/s) sum_B |cell| / mu_r) I + alpha^3/4 o~^T K(s) o~ (Eq. (6a)).
* One basis U for the three directions, from the truncated SVD of the
  snapshots q_i(omega_k, s_l) of all directions and all sampled parameters.

The conductivity needs no second parameter: nu = alpha^2 mu_0 omega sigma_*
(below Eq. (5)) carries sigma_* only through the product omega sigma_*, so a
conductivity scale t is the frequency omega t, the s_sigma of the sweep.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import tsvd


@dataclass
class MuModel:
    K_out: np.ndarray   # r x r   U^H (K - K_in) U
    K_in: np.ndarray    # r x r   U^H K_in U
    C: np.ndarray       # r x r   U^H C U
    Me: np.ndarray      # r x r   U^H (eps M) U
    Bx: np.ndarray      # r x 3   U^H C x
    BV: np.ndarray      # r x m   U^H C V
    Sv_out: np.ndarray  # m x m   V^H (K - K_in) V
    Sv_in: np.ndarray   # m x m   V^H K_in V
    Mv: np.ndarray      # m x m   V^H (eps_s M_Omega) V
    kv_out: np.ndarray  # m x 3   V^H (K x - K_in x)   (boundary columns of K included)
    kv_in: np.ndarray   # m x 3   V^H K_in x
    cxx: np.ndarray     # 3 x 3   x^T C x
    cvx: np.ndarray     # m x 3   V^H C x
    cvv: np.ndarray     # m x m   V^H C V
    nB: float           # alpha^3 |B|
    mB: float           # alpha^3 sum_B |cell| / mu_r
    alpha: float
    G_ext: np.ndarray | None = None   # Gram of [C x | C V | (K_out + eps M) U | K_in U | C U] in X^-1
    alpha_lb: float = 1.0 / np.sqrt(2.0)

    @property
    def r(self) -> int:
        return self.K_out.shape[0]

    @property
    def m(self) -> int:
        return self.Sv_out.shape[0]


def bases(D_list, O_list, tol_sigma: float = 1e-10, tol_static: float = 1e-10,
          r_max: int | None = None):
    """U from the (3, N, n_w) snapshot stacks of every sampled s (one TSVD of all their
    columns), V from the (3, N) static snapshots o~(s_l) (one TSVD, real)."""
    D = np.concatenate([np.concatenate(list(Dl), axis=1) for Dl in D_list], axis=1)
    U = tsvd.truncated_svd(D, tol_sigma, r_max)[0]
    O = np.concatenate([np.asarray(Ol).T for Ol in O_list], axis=1)
    V = tsvd.truncated_svd(O, tol_static)[0]
    return U, V


def project(problem, U: np.ndarray, V: np.ndarray) -> MuModel:
    """Galerkin projections of the parameter-independent parts (problem at s = 1, built
    with mu_split=True)."""
    K_in = problem.K_in
    K_out = problem.K - K_in
    C = problem.C
    x = problem.x
    UH = U.conj().T
    VH = V.conj().T
    kx_out = problem.kx - problem.kx_in
    a3 = problem.alpha ** 3
    return MuModel(
        K_out=UH @ (K_out @ U), K_in=UH @ (K_in @ U), C=UH @ (C[:, None] * U),
        Me=UH @ ((problem.eps * problem.M)[:, None] * U),
        Bx=UH @ (C[:, None] * x.T), BV=UH @ (C[:, None] * V),
        Sv_out=VH @ (K_out @ V), Sv_in=VH @ (K_in @ V),
        Mv=VH @ ((problem.eps_static * problem.M_omega)[:, None] * V),
        kv_out=VH @ kx_out.T, kv_in=VH @ problem.kx_in.T,
        cxx=x @ (C[:, None] * x.T), cvx=VH @ (C[:, None] * x.T), cvv=VH @ (C[:, None] * V),
        nB=a3 * problem.vol_B, mB=a3 * problem.vol_B_mu, alpha=problem.alpha)


def attach_extended_gram(model: MuModel, problem, U: np.ndarray, V: np.ndarray, X_diag: np.ndarray) -> None:
    """The certificate of Lemma 4.2 at a permeability scale s.  The residual of direction i,
    r_i = i w C o_i(s) - (K(s) + eps M - i w C) U p_i with the reduced o_i(s) = x_i + V y_i(s),
    is Phi_ext w_i for Phi_ext = [C x | C V | (K_out + eps M) U | K_in U | C U] and
    w_i = [i w e_i ; i w y_i ; -p_i ; -p_i / s ; i w p_i]; G_ext = Phi_ext^H X^-1 Phi_ext."""
    C = problem.C
    K_in = problem.K_in
    K_out = problem.K - K_in
    Phi = np.concatenate([C[:, None] * problem.x.T, C[:, None] * V,
                          K_out @ U + (problem.eps * problem.M)[:, None] * U, K_in @ U, C[:, None] * U], axis=1)
    model.G_ext = Phi.conj().T @ (Phi / np.asarray(X_diag)[:, None])


def certificate(model: MuModel, omegas, s_mu: float = 1.0, s_sigma: float = 1.0) -> np.ndarray:
    """(Delta[omega])_ij of Lemma 4.2 at the scale s_mu, shape (n_w, 3, 3):
    ||r^_i||^2 = w_i^H G_ext w_i and Delta_ij = alpha^3 / (8 alpha_LB) (||r^_i||^2 + ||r^_j||^2
    + ||r^_i - r^_j||^2)."""
    w_all = np.asarray(omegas, dtype=np.float64) * s_sigma
    st = static_state(model, s_mu)
    K = model.K_out + model.K_in / s_mu
    a3 = model.alpha ** 3
    out = np.empty((w_all.size, 3, 3))
    for n, w in enumerate(w_all):
        P = np.linalg.solve(K + model.Me - 1j * w * model.C, 1j * w * st["B"])
        W = [np.concatenate([1j * w * np.eye(3)[i], 1j * w * st["y"][:, i], -P[:, i], -P[:, i] / s_mu,
                             1j * w * P[:, i]]) for i in range(3)]
        GW = [model.G_ext @ W[j] for j in range(3)]
        nrm = np.array([np.real(np.vdot(W[i], GW[i])) for i in range(3)])
        for i in range(3):
            for j in range(3):
                diff = nrm[i] + nrm[j] - 2.0 * np.real(np.vdot(W[i], GW[j]))
                out[n, i, j] = a3 / (8.0 * model.alpha_lb) * (nrm[i] + nrm[j] + diff)
    return out


def certificate_term_scale(model: MuModel, omegas, s_mu: float = 1.0, s_sigma: float = 1.0) -> np.ndarray:
    """Per frequency alpha^3 / (4 alpha_LB) max_i |w_i|^T |G_ext| |w_i|: the size of the terms the
    Gram form of the certificate sums (Delta cancels them at an accurate model), the scale its
    rounding is measured against."""
    w_all = np.asarray(omegas, dtype=np.float64) * s_sigma
    st = static_state(model, s_mu)
    K = model.K_out + model.K_in / s_mu
    absG = np.abs(model.G_ext)
    out = np.empty(w_all.size)
    for n, w in enumerate(w_all):
        P = np.linalg.solve(K + model.Me - 1j * w * model.C, 1j * w * st["B"])
        W = [np.abs(np.concatenate([1j * w * np.eye(3)[i], 1j * w * st["y"][:, i], -P[:, i], -P[:, i] / s_mu,
                                    1j * w * P[:, i]])) for i in range(3)]
        out[n] = model.alpha ** 3 / (4.0 * model.alpha_lb) * max(x @ absG @ x for x in W)
    return out


def residual_norms_direct(model: MuModel, problem, U: np.ndarray, V: np.ndarray, X_diag: np.ndarray,
                          omega: float, s_mu: float) -> np.ndarray:
    """||r^_i||^2 from the full-order residual vector of the problem at scale s_mu (pin for the
    Gram form): r_i = i w C (x_i + V y_i(s)) - A(w, s) U p_i."""
    st = static_state(model, s_mu)
    K = problem.K - problem.K_in + problem.K_in / s_mu
    A = (sp.csc_matrix(K, dtype=np.complex128) + sp.diags(problem.eps * problem.M - 1j * omega * problem.C))
    P = np.linalg.solve(model.K_out + model.K_in / s_mu + model.Me - 1j * omega * model.C, 1j * omega * st["B"])
    o = problem.x + np.real(V @ st["y"]).T
    out = np.empty(3)
    for i in range(3):
        rho = 1j * omega * problem.C * o[i] - A @ (U @ P[:, i])
        out[i] = np.real(np.vdot(rho, rho / X_diag))
    return out


def residual_differences_direct(model: MuModel, problem, U: np.ndarray, V: np.ndarray, X_diag: np.ndarray,
                                omega: float, s_mu: float) -> np.ndarray:
    """||r^_i - r^_j||^2 for every pair (i, j) from the explicit full-order residual vectors of the
    problem at scale s_mu (pin for the off-diagonal entries of Lemma 4.2)."""
    st = static_state(model, s_mu)
    K = problem.K - problem.K_in + problem.K_in / s_mu
    A = (sp.csc_matrix(K, dtype=np.complex128) + sp.diags(problem.eps * problem.M - 1j * omega * problem.C))
    P = np.linalg.solve(model.K_out + model.K_in / s_mu + model.Me - 1j * omega * model.C, 1j * omega * st["B"])
    o = problem.x + np.real(V @ st["y"]).T
    rho = [1j * omega * problem.C * o[i] - A @ (U @ P[:, i]) for i in range(3)]
    out = np.empty((3, 3))
    for i in range(3):
        for j in range(3):
            d = rho[i] - rho[j]
            out[i, j] = np.real(np.vdot(d, d / X_diag))
    return out


def static_state(model: MuModel, s: float):
    """y(s), b(s), c00(s), N0(s) and their derivatives with respect to s.

    Returns dict with y, dy (m x 3), B, dB (r x 3), c00, dc00, N0, dN0 (3 x 3)."""
    S = model.Sv_out + model.Sv_in / s + model.Mv
    rhs = -(model.kv_out + model.kv_in / s)
    y = np.linalg.solve(S, rhs)
    # d/ds of S y = rhs:  S dy = d(rhs) - dS y,  dS = -Sv_in / s^2,  d(rhs) = kv_in / s^2
    dy = np.linalg.solve(S, (model.kv_in + model.Sv_in @ y) / s ** 2)
    B = model.Bx + model.BV @ y
    dB = model.BV @ dy
    cross = model.cvx.conj().T @ y                       # [i, j] = (V^H C x_i)^H y_j
    c00 = model.cxx + np.real(cross + cross.conj().T + y.conj().T @ model.cvv @ y)
    dcross = model.cvx.conj().T @ dy
    q = dy.conj().T @ model.cvv @ y
    dc00 = np.real(dcross + dcross.conj().T + q + q.conj().T)
    Kv = model.Sv_out + model.Sv_in / s
    a3 = model.alpha ** 3
    N0 = (model.nB - model.mB / s) * np.eye(3) + a3 / 4.0 * np.real(y.conj().T @ Kv @ y)
    qk = dy.conj().T @ Kv @ y
    dN0 = (model.mB / s ** 2) * np.eye(3) + a3 / 4.0 * np.real(
        qk + qk.conj().T - y.conj().T @ model.Sv_in @ y / s ** 2)
    return dict(y=y, dy=dy, B=B, dB=dB, c00=c00, dc00=dc00, N0=N0, dN0=dN0)


def signature(model: MuModel, omegas, s_mu: float = 1.0, s_sigma: float = 1.0):
    """R~ (with N0) and I at the frequencies omegas for the parameter s_mu, with a
    conductivity scale s_sigma; shapes (n_w, 3, 3).  Dense solves per frequency."""
    w = np.asarray(omegas, dtype=np.float64) * s_sigma
    st = static_state(model, s_mu)
    K = model.K_out + model.K_in / s_mu
    A = (K + model.Me)[None] - 1j * w[:, None, None] * model.C[None]
    P = np.linalg.solve(A, (1j * w)[:, None, None] * st["B"][None])
    PH = np.conj(np.swapaxes(P, 1, 2))
    a3 = model.alpha ** 3
    R = st["N0"][None] - a3 / 4.0 * np.real(PH @ K @ P)
    BH = st["B"].conj().T
    F = st["c00"][None] + np.real(PH @ model.C @ P + BH[None] @ P + PH @ st["B"][None])
    I = w[:, None, None] * a3 / 4.0 * F
    return R, I


def tangent_s_mu(model: MuModel, omegas, s_mu: float = 1.0, s_sigma: float = 1.0):
    """dR~/ds_mu and dI/ds_mu (forward mode, dense): K(s), b(s), c00(s) and N0(s) all vary."""
    w = np.asarray(omegas, dtype=np.float64) * s_sigma
    st = static_state(model, s_mu)
    K = model.K_out + model.K_in / s_mu
    dK = -model.K_in / s_mu ** 2
    A = (K + model.Me)[None] - 1j * w[:, None, None] * model.C[None]
    P = np.linalg.solve(A, (1j * w)[:, None, None] * st["B"][None])
    dP = np.linalg.solve(A, (1j * w)[:, None, None] * st["dB"][None] - dK[None] @ P)
    PH = np.conj(np.swapaxes(P, 1, 2))
    dPH = np.conj(np.swapaxes(dP, 1, 2))
    a3 = model.alpha ** 3
    dR = st["dN0"][None] - a3 / 4.0 * np.real(dPH @ K @ P + PH @ K @ dP + PH @ dK @ P)
    B, dB = st["B"], st["dB"]
    dF = st["dc00"][None] + np.real(dPH @ model.C @ P + PH @ model.C @ dP + dB.conj().T[None] @ P
                                    + B.conj().T[None] @ dP + dPH @ B[None] + PH @ dB[None])
    dI = w[:, None, None] * a3 / 4.0 * dF
    return dR, dI
