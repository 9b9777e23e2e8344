"""ctypes declarations of include/mrom.h and library loading."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmrom.so")
_LIB = None

STATUS = {0: "MROM_OK", 1: "MROM_EINVAL", 2: "MROM_ENOMEM", 3: "MROM_ECUDA", 4: "MROM_ESINGULAR",
          5: "MROM_ENOTCONVERGED", 6: "MROM_ETIMEOUT", 7: "MROM_ECALLBACK", 8: "MROM_ENOTSUP"}

# Every function the header declares (checked by tests/test_abi.py).
EXPORTS = [
    "mrom_create", "mrom_destroy", "mrom_set_stream", "mrom_synchronize", "mrom_last_error",
    "mrom_launch_count", "mrom_rom_from_reduced", "mrom_rom_rank", "mrom_rom_free", "mrom_sweep",
    "mrom_certificate", "mrom_plan_create", "mrom_plan_sweep", "mrom_plan_destroy", "mrom_tune",
    "mrom_sweep_noalloc", "mrom_project", "mrom_rom_get", "mrom_adapt", "mrom_sweep_vjp", "mrom_sweep_mixed",
    "mrom_project_dirs", "mrom_set_projection_precision", "mrom_set_solver", "mrom_plan_solver_counts",
    "mrom_plan_timing", "mrom_rom_from_reduced_batch", "mrom_invariants", "mrom_project_mu",
    "mrom_rom_static_rank", "mrom_rom_mu_state", "mrom_fom_solve", "mrom_rom_from_packed", "mrom_rom_free_batch",
    "mrom_fp64_peak", "mrom_static_solve", "mrom_plan_sweep_invariants", "mrom_sweep_host",
    "mrom_tune_pencil",
]


class MromError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class mrom_fom(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("K_rowptr", ctypes.c_void_p),
        ("K_col", ctypes.c_void_p),
        ("K_val", ctypes.c_void_p),
        ("C_diag", ctypes.c_void_p),
        ("M_diag", ctypes.c_void_p),
        ("eps", ctypes.c_double),
        ("o", ctypes.c_void_p),
        ("X_diag", ctypes.c_void_p),
        ("alpha", ctypes.c_double),
        ("alpha_lb", ctypes.c_double),
        ("vol_B", ctypes.c_double),
        ("N0", ctypes.c_void_p),
        ("X_rowptr", ctypes.c_void_p),
        ("X_col", ctypes.c_void_p),
        ("X_val", ctypes.c_void_p),
        ("X_tol", ctypes.c_double),
        ("X_max_iter", ctypes.c_int32),
    ]


class mrom_packed_obj(ctypes.Structure):
    _fields_ = [
        ("r", ctypes.c_int32),
        ("has_kin", ctypes.c_int32),
        ("has_me", ctypes.c_int32),
        ("has_gram", ctypes.c_int32),
        ("offset", ctypes.c_int64),
        ("c00", ctypes.c_double * 9),
        ("N0", ctypes.c_double * 9),
        ("alpha", ctypes.c_double),
        ("alpha_lb", ctypes.c_double),
        ("vol_B", ctypes.c_double),
    ]


class mrom_fom_mu(ctypes.Structure):
    _fields_ = [
        ("Kin_rowptr", ctypes.c_void_p),
        ("Kin_col", ctypes.c_void_p),
        ("Kin_val", ctypes.c_void_p),
        ("x", ctypes.c_void_p),
        ("kx", ctypes.c_void_p),
        ("kx_in", ctypes.c_void_p),
        ("M_static", ctypes.c_void_p),
        ("vol_B_mu", ctypes.c_double),
        ("O", ctypes.c_void_p),
        ("ldo", ctypes.c_int64),
        ("n_o", ctypes.c_int32),
        ("tol_static", ctypes.c_double),
    ]


class mrom_adapt_opts(ctypes.Structure):
    _fields_ = [
        ("tol_sigma", ctypes.c_double),
        ("tol_delta", ctypes.c_double),
        ("n_star", ctypes.c_int32),
        ("max_k", ctypes.c_int32),
        ("r_max", ctypes.c_int32),
        ("theta", ctypes.c_double),
    ]


SNAPSHOT_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                               ctypes.c_void_p)


class mrom_reduced_desc(ctypes.Structure):
    _fields_ = [
        ("r", ctypes.c_int32),
        ("K", ctypes.c_void_p),
        ("K_in", ctypes.c_void_p),
        ("C", ctypes.c_void_p),
        ("Me", ctypes.c_void_p),
        ("B", ctypes.c_void_p),
        ("c00", ctypes.POINTER(ctypes.c_double)),
        ("G", ctypes.c_void_p),
        ("N0", ctypes.POINTER(ctypes.c_double)),
        ("alpha", ctypes.c_double),
        ("alpha_lb", ctypes.c_double),
        ("vol_B", ctypes.c_double),
        ("r_dirs", ctypes.c_int32 * 3),
    ]


def _declare(L):
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "mrom_create": (ctypes.c_int, [ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "mrom_destroy": (ctypes.c_int, [vp]),
        "mrom_set_stream": (ctypes.c_int, [vp, vp]),
        "mrom_synchronize": (ctypes.c_int, [vp]),
        "mrom_last_error": (ctypes.c_char_p, [vp]),
        "mrom_launch_count": (i64, [vp]),
        "mrom_set_projection_precision": (ctypes.c_int, [vp, ctypes.c_int]),
        "mrom_set_solver": (ctypes.c_int, [vp, ctypes.c_int]),
        "mrom_plan_timing": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]),
        "mrom_rom_from_reduced_batch": (ctypes.c_int, [vp, ctypes.c_int32, vp, vp]),
        "mrom_invariants": (ctypes.c_int, [vp, vp, i64, vp]),
        "mrom_static_solve": (ctypes.c_int, [vp, ctypes.POINTER(mrom_fom), vp, i64, vp, vp, vp, vp, vp, vp, vp, i32,
                                             ctypes.c_double, i32, vp, ctypes.POINTER(i32)]),
        "mrom_plan_sweep_invariants": (ctypes.c_int, [vp, vp, i32, vp, vp, vp, vp]),
        "mrom_fp64_peak": (ctypes.c_int, [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "mrom_plan_solver_counts": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "mrom_rom_from_reduced": (ctypes.c_int, [vp, ctypes.POINTER(mrom_reduced_desc), ctypes.POINTER(vp)]),
        "mrom_rom_rank": (i32, [vp]),
        "mrom_rom_static_rank": (i32, [vp]),
        "mrom_rom_free_batch": (None, [ctypes.POINTER(vp), i32]),
        "mrom_rom_from_packed": (ctypes.c_int, [vp, i32, ctypes.POINTER(mrom_packed_obj), vp, ctypes.c_size_t,
                                                ctypes.POINTER(vp)]),
        "mrom_sweep_host": (ctypes.c_int, [vp, i32, ctypes.POINTER(mrom_packed_obj), vp, ctypes.c_size_t, vp, i32,
                                           vp, vp, vp, i32]),
        "mrom_fom_solve": (ctypes.c_int, [vp, ctypes.POINTER(mrom_fom), ctypes.POINTER(ctypes.c_double), i32,
                                          ctypes.c_double, i32, vp, i64, ctypes.POINTER(i32),
                                          ctypes.POINTER(ctypes.c_double)]),
        "mrom_rom_mu_state": (ctypes.c_int, [vp, ctypes.c_double, vp, dp, dp, vp, dp, dp]),
        "mrom_project_mu": (ctypes.c_int, [vp, ctypes.POINTER(mrom_fom), ctypes.POINTER(mrom_fom_mu), vp, i64, i32,
                                           ctypes.c_double, i32, ctypes.POINTER(vp), ctypes.POINTER(i32),
                                           ctypes.POINTER(i32)]),
        "mrom_rom_free": (None, [vp]),
        "mrom_sweep": (ctypes.c_int, [vp, ctypes.POINTER(vp), i32, dp, i32, i32, dp, dp, dp, dp, dp]),
        "mrom_certificate": (ctypes.c_int, [vp, ctypes.POINTER(vp), i32, dp, i32, i32, dp]),
        "mrom_plan_create": (ctypes.c_int, [vp, ctypes.POINTER(vp), i32, i32, ctypes.POINTER(vp)]),
        "mrom_plan_sweep": (ctypes.c_int, [vp, dp, i32, dp, dp, dp]),
        "mrom_plan_destroy": (ctypes.c_int, [vp]),
        "mrom_tune": (ctypes.c_int, [vp, ctypes.POINTER(vp), i32, i32, ctypes.POINTER(i32)]),
        "mrom_tune_pencil": (ctypes.c_int, [vp, ctypes.POINTER(vp), i32, i32, ctypes.POINTER(i32)]),
        "mrom_sweep_noalloc": (ctypes.c_int, [vp, ctypes.POINTER(vp), i32, dp, i32, i32, dp, dp, dp]),
        "mrom_project": (ctypes.c_int, [vp, ctypes.POINTER(mrom_fom), vp, i64, i32, ctypes.c_double, i32, vp, i32,
                                        ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(i32)]),
        "mrom_project_dirs": (ctypes.c_int, [vp, ctypes.POINTER(mrom_fom), vp, i64, i32, ctypes.c_double, i32, vp,
                                             ctypes.POINTER(i32), ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(i32)]),
        "mrom_rom_get": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp]),
        "mrom_sweep_mixed": (ctypes.c_int, [vp, ctypes.POINTER(vp), i32, dp, i32, i32, i32, dp, dp, dp]),
        "mrom_sweep_vjp": (ctypes.c_int, [vp, ctypes.POINTER(vp), i32, dp, i32, i32, dp, dp, dp, dp, dp, dp, dp, dp,
                                          dp]),
        "mrom_adapt": (ctypes.c_int, [vp, ctypes.POINTER(mrom_fom), ctypes.POINTER(ctypes.c_double), i32, vp,
                                      SNAPSHOT_CB, vp, dp, i32, ctypes.POINTER(mrom_adapt_opts),
                                      ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def lib():
    """Load libmrom.so (built by paper_2307_05590_gb300/build.py); raise if it is missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise MromError(3, f"{LIB_PATH} not built; run paper_2307_05590_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        _declare(L)
        _LIB = L
    return _LIB


def check(status: int, handle) -> None:
    if status != 0:
        msg = lib().mrom_last_error(handle).decode() if handle else ""
        raise MromError(status, msg)
