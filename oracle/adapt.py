"""Adaptive snapshot selection, Algorithm 1 (Sect. 4.4).

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.

Readings where the algorithm leaves details open:
* certificates are evaluated on the output frequency grid;
* interval n is [omega_n, omega_{n+1}) over the sorted snapshot frequencies,
  and grid points equal to an existing snapshot are not candidates;
* the candidate of an interval is the grid point where max_ij Delta_ij is
  largest (ties: lowest omega); the N_* intervals with the largest Lambda_n
  each contribute one new snapshot (at most one per interval);
* the variant with a threshold 0 < theta <= 1 (Sect. 4.4, after Algorithm 1)
  takes the candidates of every interval with Lambda_n >= theta Lambda, again
  one per interval, the largest Lambda_n first and at most N_* of them per
  iteration (so that the snapshot count stays bounded); theta = 0 is the
  fixed-N_* rule;
* |B_alpha| = alpha^3 |B|;
* the loop stops as soon as Lambda / |B_alpha| <= TOL_Delta, before computing
  further snapshots, or when k reaches MAX_k.
"""
from __future__ import annotations

import numpy as np

from . import certificate, pipeline, rom


def interval_maxima(snaps: np.ndarray, omega_out: np.ndarray, dmax: np.ndarray):
    """Lambda_n and its arg-max frequency for every snapshot interval."""
    snaps = np.sort(snaps)
    lam = np.full(snaps.size - 1, -np.inf)
    cand = np.full(snaps.size - 1, np.nan)
    is_snap = np.isin(omega_out, snaps)
    for n in range(snaps.size - 1):
        m = (omega_out >= snaps[n]) & (omega_out < snaps[n + 1]) & ~is_snap
        if not np.any(m):
            continue
        idx = np.flatnonzero(m)
        k = idx[np.argmax(dmax[idx])]          # first maximum -> lowest omega
        lam[n] = dmax[k]
        cand[n] = omega_out[k]
    return lam, cand


def select_new(lam_n: np.ndarray, cand: np.ndarray, n_star: int, theta: float = 0.0) -> np.ndarray:
    """New snapshot frequencies (ascending) from the interval maxima: the intervals in
    decreasing order of Lambda_n (ties: lower interval first), at most n_star of them, and
    with theta > 0 only those with Lambda_n >= theta max_n Lambda_n."""
    lam = float(np.max(lam_n))
    order = np.argsort(-lam_n, kind="stable")
    keep = [n for n in order if np.isfinite(lam_n[n]) and (theta <= 0.0 or lam_n[n] >= theta * lam)]
    return np.sort(cand[keep[:n_star]])


def adaptive_podp(problem, snapshot_fn, omega0, omega_out, *, tol_sigma=1e-6, tol_delta=1e-3,
                  n_star=2, max_k=10, r_max=None, shared=False, X_diag=None, theta=0.0):
    """Run Algorithm 1; returns (model, snapshot omegas, Lambda history, k).

    snapshot_fn(omegas) must return the (3, N, len(omegas)) full-order
    solutions at those frequencies (the initial and the added full-order snapshots).
    """
    omega_out = np.asarray(omega_out, dtype=np.float64)
    snaps = np.asarray(omega0, dtype=np.float64)
    D = snapshot_fn(snaps)
    omega_min = float(omega_out.min())
    model, _, _ = pipeline.build_model(problem, D, tol_sigma=tol_sigma, r_max=r_max, shared=shared,
                                       omega_min=omega_min, X_diag=X_diag)
    b_alpha = problem.alpha ** 3 * problem.vol_B
    k, Lam, hist = 1, np.inf, []
    while Lam / b_alpha > tol_delta and k < max_k:
        k += 1
        P = rom.reduced_solve(model, omega_out)
        Delta = certificate.certificate(model, omega_out, P)
        lam_n, cand = interval_maxima(snaps, omega_out, Delta.max(axis=(1, 2)))
        Lam = float(np.max(lam_n))
        hist.append(Lam)
        if Lam / b_alpha <= tol_delta:
            break
        new = select_new(lam_n, cand, n_star, theta)
        D = np.concatenate([D, snapshot_fn(new)], axis=2)
        snaps = np.concatenate([snaps, new])
        model, _, _ = pipeline.build_model(problem, D, tol_sigma=tol_sigma, r_max=r_max,
                                           shared=shared, omega_min=omega_min, X_diag=X_diag)
    return model, np.sort(snaps), hist, k
