"""Derivatives of the reduced tensors with respect to omega, s_sigma and s_mu.

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.

For a shared-basis reduced object with a conductivity scale s_sigma and a
permeability scale s_mu (K(s_mu) = K_out + K_in / s_mu):
  A = K(s_mu) - i omega s_sigma C,  A P = i omega s_sigma B,
  R = -alpha^3/4 Re(P^H K(s_mu) P),
  I = omega s_sigma alpha^3/4 (c00 + Re(P^H C P + B^H P + P^H B)),
which is Eqs. (17)-(19) with C, b and c00 scaled by s_sigma (nu is linear in
sigma, Sect. 3 below Eq. (5)).  Tangents follow from
dP = A^-1 (d(rhs) - dA P) (forward mode, dense); the VJP contracts them with
output cotangents.  Parity unpinned against the paper (the paper has no
gradients); pinned by central finite differences and by the exact identity
d/ds_sigma = omega d/domega at s_sigma = 1.
"""
from __future__ import annotations

import numpy as np


def _solve(obj, w, s_sigma, s_mu):
    K = obj.K_out + obj.K_in / s_mu
    A = K[None] - 1j * (w * s_sigma)[:, None, None] * obj.C[None]
    rhs = (1j * w * s_sigma)[:, None, None] * obj.B[None]
    return K, A, np.linalg.solve(A, rhs)


def forward(obj, omegas, s_sigma=1.0, s_mu=1.0):
    """R, I of shape (n_w, 3, 3)."""
    w = np.asarray(omegas, dtype=np.float64)
    K, A, P = _solve(obj, w, s_sigma, s_mu)
    a3 = obj.alpha ** 3
    PH = np.conj(np.swapaxes(P, 1, 2))
    R = -a3 / 4.0 * np.real(PH @ K @ P)
    BH = obj.B.conj().T
    F = obj.c00[None] + np.real(PH @ obj.C @ P + BH[None] @ P + PH @ obj.B[None])
    I = (w * s_sigma)[:, None, None] * a3 / 4.0 * F
    return R, I


def tangents(obj, omegas, s_sigma=1.0, s_mu=1.0):
    """dR/dtheta, dI/dtheta for theta in (omega, s_sigma, s_mu): arrays (3, n_w, 3, 3)."""
    w = np.asarray(omegas, dtype=np.float64)
    K, A, P = _solve(obj, w, s_sigma, s_mu)
    a3 = obj.alpha ** 3
    PH = np.conj(np.swapaxes(P, 1, 2))
    BH = obj.B.conj().T
    F = obj.c00[None] + np.real(PH @ obj.C @ P + BH[None] @ P + PH @ obj.B[None])
    nw = w.size
    dK_mu = -obj.K_in / s_mu ** 2
    cases = [
        # (dA, d rhs, dK, d(omega s_sigma))
        (-1j * s_sigma * np.broadcast_to(obj.C, (nw,) + obj.C.shape),
         1j * s_sigma * np.broadcast_to(obj.B, (nw,) + obj.B.shape), None, np.full(nw, s_sigma)),
        (-1j * w[:, None, None] * obj.C[None], 1j * w[:, None, None] * obj.B[None], None, w),
        (np.broadcast_to(dK_mu, (nw,) + dK_mu.shape), np.zeros_like(P), dK_mu, np.zeros(nw)),
    ]
    dR = np.empty((3, nw, 3, 3))
    dI = np.empty((3, nw, 3, 3))
    for t, (dA, drhs, dK, dws) in enumerate(cases):
        dP = np.linalg.solve(A, drhs - dA @ P)
        dPH = np.conj(np.swapaxes(dP, 1, 2))
        g = dPH @ K @ P + PH @ K @ dP
        if dK is not None:
            g = g + PH @ dK @ P
        dR[t] = -a3 / 4.0 * np.real(g)
        dF = np.real(dPH @ obj.C @ P + PH @ obj.C @ dP + BH[None] @ dP + dPH @ obj.B[None])
        dI[t] = a3 / 4.0 * (dws[:, None, None] * F + (w * s_sigma)[:, None, None] * dF)
    return dR, dI


def vjp(obj, omegas, gR, gI, s_sigma=1.0, s_mu=1.0):
    """Vector-Jacobian product: (g_omega[n_w], g_s_sigma, g_s_mu)."""
    dR, dI = tangents(obj, omegas, s_sigma, s_mu)
    contrib = np.einsum("twij,wij->tw", dR, gR) + np.einsum("twij,wij->tw", dI, gI)
    return contrib[0], float(contrib[1].sum()), float(contrib[2].sum())


def central_difference(obj, omegas, which: int, h_rel: float = 1e-6, s_sigma=1.0, s_mu=1.0):
    """Central finite difference of (R, I) in omega (per point), s_sigma or s_mu."""
    w = np.asarray(omegas, dtype=np.float64)
    if which == 0:
        h = h_rel * w
        Rp, Ip = forward(obj, w + h, s_sigma, s_mu)
        Rm, Im = forward(obj, w - h, s_sigma, s_mu)
        return (Rp - Rm) / (2 * h)[:, None, None], (Ip - Im) / (2 * h)[:, None, None]
    base = s_sigma if which == 1 else s_mu
    h = h_rel * base
    if which == 1:
        Rp, Ip = forward(obj, w, s_sigma + h, s_mu)
        Rm, Im = forward(obj, w, s_sigma - h, s_mu)
    else:
        Rp, Ip = forward(obj, w, s_sigma, s_mu + h)
        Rm, Im = forward(obj, w, s_sigma, s_mu - h)
    return (Rp - Rm) / (2 * h), (Ip - Im) / (2 * h)
