"""Helpers shared by the GPU parity tests (oracle side + tolerances)."""
import numpy as np

from oracle import certificate, rom


def oracle_sweep(obj, omegas, s_sigma=1.0):
    """R, I, Delta and the per-(omega) term scales from the CPU oracle."""
    return oracle_model_sweep(rom.from_reduced_object(obj), omegas, s_sigma)


def oracle_model_sweep(model, omegas, s_sigma=1.0):
    """As oracle_sweep, for a shared-basis oracle ReducedModel."""
    w = np.asarray(omegas, dtype=np.float64) * s_sigma
    P = rom.reduced_solve(model, w)
    R, I = rom.mm_tensors(model, w, P)
    Dl = certificate.certificate(model, w, P) if model.gram is not None else None
    a3 = model.alpha ** 3
    sI = np.empty(w.size)
    sD = np.empty(w.size)
    absG = np.abs(model.gram) if model.gram is not None else None
    C = model.C[0][0]
    B = np.stack([model.b(i) for i in range(3)], 1)
    for n in range(w.size):
        Pm = np.stack([P[i][n] for i in range(3)], 1)
        hc = np.abs(Pm.conj().T @ C @ Pm).max()
        bp = np.abs(B.conj().T @ Pm).max()
        sI[n] = w[n] * a3 / 4 * (np.abs(model.c00).max() + hc + 2 * bp)
        if absG is not None:
            W = certificate.residual_weights(model, w[n], [P[i][n] for i in range(3)])
            sD[n] = a3 / (4 * model.alpha_lb) * max(np.abs(x) @ absG @ np.abs(x) for x in W)
    return R, I, Dl, sI, sD


def rel_errors(Rg, Ig, Dg, R, I, Dl, sI, sD):
    """Normwise errors per frequency: R against max|R|, I and Delta against their term scales."""
    eR = np.abs(Rg - R).reshape(len(R), -1).max(1) / np.abs(R).reshape(len(R), -1).max(1)
    eI = np.abs(Ig - I).reshape(len(I), -1).max(1) / sI
    eD = np.abs(Dg - Dl).reshape(len(Dl), -1).max(1) / sD if Dg is not None else np.zeros(1)
    return eR.max(), eI.max(), eD.max()
