"""Helpers shared by the GPU parity tests (oracle side + tolerances)."""
import numpy as np

from oracle import certificate, rom


def oracle_sweep(obj, omegas, s_sigma=1.0):
    """R, I, Delta and the per-(omega) term scales from the CPU oracle."""
    w = np.asarray(omegas, dtype=np.float64) * s_sigma
    model = rom.from_reduced_object(obj)
    P = rom.reduced_solve(model, w)
    R, I = rom.mm_tensors(model, w, P)
    Dl = certificate.certificate(model, w, P)
    a3 = obj.alpha ** 3
    sI = np.empty(w.size)
    sD = np.empty(w.size)
    absG = np.abs(obj.G)
    for n in range(w.size):
        Pm = np.stack([P[i][n] for i in range(3)], 1)
        hc = np.abs(Pm.conj().T @ obj.C @ Pm).max()
        bp = np.abs(obj.B.conj().T @ Pm).max()
        sI[n] = w[n] * a3 / 4 * (np.abs(obj.c00).max() + hc + 2 * bp)
        W = certificate.residual_weights(model, w[n], [P[i][n] for i in range(3)])
        sD[n] = a3 / (4 * obj.alpha_lb) * max(np.abs(x) @ absG @ np.abs(x) for x in W)
    return R, I, Dl, sI, sD


def rel_errors(Rg, Ig, Dg, R, I, Dl, sI, sD):
    """Normwise errors per frequency: R against max|R|, I and Delta against their term scales."""
    eR = np.abs(Rg - R).reshape(len(R), -1).max(1) / np.abs(R).reshape(len(R), -1).max(1)
    eI = np.abs(Ig - I).reshape(len(I), -1).max(1) / sI
    eD = np.abs(Dg - Dl).reshape(len(Dl), -1).max(1) / sD if Dg is not None else np.zeros(1)
    return eR.max(), eI.max(), eD.max()
