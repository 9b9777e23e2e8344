"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package defines *problems*, not the reduced-order method: structured
FIT (finite integration) stand-ins for the paper's hp-FEM matrices K, C, M
(Sect. 3.1, Eq. (10)), the static theta^(0) data, full-order snapshot
matrices D_i (Eq. (13)), and synthetic reduced dictionaries for the batched
sweep.  Nothing here performs a truncated SVD, a projection, a reduced solve,
a tensor post-processing formula or a certificate; those belong to the oracle
(``oracle/``) and to the CUDA library.
"""
from .fit import FitProblem, fit_problem, CUBE_C1, CUBE_C2, TWO_MATERIAL_C5
from .snapshots import full_order_snapshots, synthetic_snapshot_matrix
from .dictionary import ReducedObject, reduced_dictionary, reduced_object
from .grids import log_omegas

__all__ = [
    "FitProblem", "fit_problem", "CUBE_C1", "CUBE_C2", "TWO_MATERIAL_C5",
    "full_order_snapshots", "synthetic_snapshot_matrix",
    "ReducedObject", "reduced_dictionary", "reduced_object", "log_omegas",
]
