"""Off-line stage of PODP end to end: snapshots -> TSVD -> projection -> Gram.

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use it.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import certificate, rom, tsvd


def build_model(problem, D: np.ndarray, *, tol_sigma: float = 1e-6, r_max: int | None = None,
                shared: bool = False, with_gram: bool = True, omega_min: float = 10.0,
                eps_in_R: bool = False, X_diag: np.ndarray | None = None):
    """ReducedModel from the (3, N, N_s) snapshot stack D (Sect. 4.1-4.3, Lemma 4.2).

    shared=False: one TSVD per direction (Eq. (15) for D_1, D_2, D_3).
    shared=True:  one TSVD of [D_1 D_2 D_3] used for all three directions.
    X_diag: a diagonal certificate inner product instead of K + eps M + omega_min C.
    """
    if shared:
        U, s, _, s_all = tsvd.truncated_svd(np.concatenate(list(D), axis=1), tol_sigma, r_max)
        bases = U
        sv = [s_all]
    else:
        bases, sv = [], []
        for i in range(3):
            U, s, _, s_all = tsvd.truncated_svd(D[i], tol_sigma, r_max)
            bases.append(U)
            sv.append(s_all)
    model = rom.project(problem, bases, eps_in_R=eps_in_R)
    if with_gram:
        if X_diag is not None:
            X = sp.diags(np.asarray(X_diag, dtype=np.float64)).tocsc()
        else:
            X = certificate.inner_product_matrix(problem, omega_min)
        certificate.attach_gram(model, problem, bases, X)
    return model, bases, sv
