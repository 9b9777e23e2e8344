"""Python binding of libmrom (reduced-order MPT spectral signatures on GB300).

Argument marshalling only: every computation runs in the CUDA library.  The
functions keep the C names of include/mrom.h (mrom_create, mrom_sweep, ...);
array arguments are torch tensors (device tensors for compute calls; host or
device for object creation) or numpy arrays (object creation only).
Importing this module does not load the library; the first call does, and it
raises if libmrom.so has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _abi
from ._abi import MromError, lib, mrom_reduced_desc  # noqa: F401

__all__ = [
    "MromError", "lib", "Handle", "ReducedObject", "Plan",
    "mrom_create", "mrom_destroy", "mrom_synchronize", "mrom_last_error", "mrom_launch_count",
    "mrom_rom_from_reduced", "mrom_rom_free", "mrom_rom_rank", "mrom_sweep", "mrom_certificate",
    "mrom_plan_create", "mrom_plan_sweep", "mrom_plan_destroy", "mrom_tune", "mrom_sweep_noalloc",
    "FullOrder", "mrom_project", "mrom_rom_get", "mrom_adapt", "mrom_sweep_vjp", "MromSweep", "signature",
    "mrom_sweep_mixed", "mrom_project_dirs", "mrom_invariants", "mrom_fp64_peak", "mrom_static_solve", "static_solver_for", "PermeabilityData", "mrom_project_mu",
    "mrom_rom_mu_state", "mrom_fom_solve", "PackedDictionary", "mrom_sweep_host", "mrom_tune_pencil",
]


def _ptr(x) -> int:
    """Raw data pointer of a contiguous torch tensor or numpy array (0 for None)."""
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


class Handle:
    """An mrom_handle bound to a CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self._h = ctypes.c_void_p()
        _abi.check(lib().mrom_create(int(device), ctypes.c_void_p(stream), ctypes.byref(self._h)), None)
        self.device = device

    @property
    def ptr(self):
        return self._h

    def synchronize(self):
        _abi.check(lib().mrom_synchronize(self._h), self._h)

    def launch_count(self) -> int:
        return int(lib().mrom_launch_count(self._h))

    def set_solver(self, lu: bool) -> None:
        """MROM_SOLVER_LU (every object by LU elimination) or MROM_SOLVER_AUTO (pencil route
        where it is accurate) for plans and sweeps created afterwards."""
        _abi.check(lib().mrom_set_solver(self._h, 1 if lu else 0), self._h)

    def set_projection_precision(self, mixed: bool) -> None:
        """MROM_MIXED (complex64 SpMM and Gram products) or MROM_FP64 for mrom_project."""
        _abi.check(lib().mrom_set_projection_precision(self._h, 1 if mixed else 0), self._h)

    def close(self):
        if self._h:
            lib().mrom_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ReducedObject:
    """An mrom_rom_t created from reduced data (mrom_rom_from_reduced)."""

    def __init__(self, handle: Handle, r: int, K, C, B, c00, *, G=None, K_in=None, Me=None, N0=None,
                 alpha: float = 1.0, alpha_lb: float = 1.0 / np.sqrt(2.0), vol_B: float = 1.0, r_dirs=(0, 0, 0)):
        keep = [_as_c128(K), _as_c128(C), _as_c128(B), _as_f64(c00), _as_c128(G), _as_c128(K_in),
                _as_c128(Me), _as_f64(N0)]
        d = mrom_reduced_desc()
        d.r = int(r)
        d.K, d.C, d.B = _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2])
        d.c00 = ctypes.cast(_ptr(keep[3]), ctypes.POINTER(ctypes.c_double))
        d.G, d.K_in, d.Me = _ptr(keep[4]), _ptr(keep[5]), _ptr(keep[6])
        d.N0 = ctypes.cast(_ptr(keep[7]), ctypes.POINTER(ctypes.c_double)) if N0 is not None else None
        d.alpha, d.alpha_lb, d.vol_B = float(alpha), float(alpha_lb), float(vol_B)
        for i in range(3):
            d.r_dirs[i] = int(r_dirs[i])
        self._rom = ctypes.c_void_p()
        self.handle = handle
        _abi.check(lib().mrom_rom_from_reduced(handle.ptr, ctypes.byref(d), ctypes.byref(self._rom)),
                   handle.ptr)
        self.r = int(r)
        self.has_cert = G is not None

    @classmethod
    def _wrap(cls, handle: Handle, ptr, r: int, has_cert: bool):
        self = cls.__new__(cls)
        self._rom = ptr
        self.handle = handle
        self.r = int(r)
        self.has_cert = has_cert
        return self

    @classmethod
    def batch(cls, handle: Handle, items):
        """mrom_rom_from_reduced_batch: one object per dict of items (keys r, K, C, B, c00 and
        optionally G, K_in, Me, N0, alpha, alpha_lb, vol_B, r_dirs), one device allocation."""
        items = list(items)
        descs = (mrom_reduced_desc * len(items))()
        keep = []
        for d, it in zip(descs, items):
            arrs = [_as_c128(it["K"]), _as_c128(it["C"]), _as_c128(it["B"]), _as_f64(it["c00"]),
                    _as_c128(it.get("G")), _as_c128(it.get("K_in")), _as_c128(it.get("Me")),
                    _as_f64(it.get("N0"))]
            keep.append(arrs)
            d.r = int(it["r"])
            d.K, d.C, d.B = _ptr(arrs[0]), _ptr(arrs[1]), _ptr(arrs[2])
            d.c00 = ctypes.cast(_ptr(arrs[3]), ctypes.POINTER(ctypes.c_double))
            d.G, d.K_in, d.Me = _ptr(arrs[4]), _ptr(arrs[5]), _ptr(arrs[6])
            d.N0 = ctypes.cast(_ptr(arrs[7]), ctypes.POINTER(ctypes.c_double)) if arrs[7] is not None else None
            d.alpha = float(it.get("alpha", 1.0))
            d.alpha_lb = float(it.get("alpha_lb", 1.0 / np.sqrt(2.0)))
            d.vol_B = float(it.get("vol_B", 1.0))
            for i, v in enumerate(it.get("r_dirs", (0, 0, 0))):
                d.r_dirs[i] = int(v)
        out = (ctypes.c_void_p * len(items))()
        _abi.check(lib().mrom_rom_from_reduced_batch(handle.ptr, len(items), descs, out), handle.ptr)
        return [cls._wrap(handle, ctypes.c_void_p(out[k]), int(items[k]["r"]), items[k].get("G") is not None)
                for k in range(len(items))]

    @staticmethod
    def close_all(objs):
        """Release many objects with one library call (mrom_rom_free_batch)."""
        live = [o for o in objs if o._rom]
        arr = (ctypes.c_void_p * len(live))(*[o._rom.value if isinstance(o._rom, ctypes.c_void_p) else o._rom
                                              for o in live])
        lib().mrom_rom_free_batch(arr, len(live))
        for o in live:
            o._rom = ctypes.c_void_p()

    @classmethod
    def from_packed(cls, handle: Handle, packed):
        """mrom_rom_from_packed: the objects of a PackedDictionary (one copy of its buffer)."""
        n = len(packed.entries)
        out = (ctypes.c_void_p * n)()
        _abi.check(lib().mrom_rom_from_packed(handle.ptr, n, packed.entries, _ptr(packed.buffer),
                                              int(packed.nbytes), out), handle.ptr)
        return [cls._wrap(handle, ctypes.c_void_p(out[k]), int(packed.entries[k].r), bool(packed.entries[k].has_gram))
                for k in range(n)]

    @classmethod
    def from_workload_batch(cls, handle: Handle, objs, *, with_cert: bool = True):
        """Batched from_workload (one device allocation for the whole dictionary)."""
        return cls.batch(handle, [dict(r=o.r, K=o.K, C=o.C, B=o.B, c00=o.c00, G=o.G if with_cert else None,
                                       K_in=o.K_in, alpha=o.alpha, alpha_lb=o.alpha_lb, vol_B=o.vol_B)
                                  for o in objs])

    @classmethod
    def from_workload(cls, handle: Handle, obj, *, with_cert: bool = True):
        """Create from a workloads.dictionary.ReducedObject (host numpy data)."""
        return cls(handle, obj.r, obj.K, obj.C, obj.B, obj.c00, G=obj.G if with_cert else None,
                   K_in=obj.K_in, alpha=obj.alpha, alpha_lb=obj.alpha_lb, vol_B=obj.vol_B)

    @property
    def ptr(self):
        return self._rom

    def close(self):
        if self._rom:
            lib().mrom_rom_free(self._rom)
            self._rom = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as_c128(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x, dtype=np.complex128)
    import torch
    return x.to(torch.complex128).contiguous()


def _as_f64(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return np.ascontiguousarray(x, dtype=np.float64)
    import torch
    return x.to(torch.float64).contiguous()


def _rom_array(objs):
    arr = (ctypes.c_void_p * len(objs))()
    for k, o in enumerate(objs):
        arr[k] = o.ptr.value
    return arr


class PackedDictionary:
    """A dictionary laid out for mrom_rom_from_packed: every object's K, [K_in], C, [Me], B, [G]
    (complex128 row-major) back to back at 16-byte aligned offsets of one host buffer (pinned
    when pin=True and torch is available), with the per-object records."""

    def __init__(self, items, *, pin: bool = True):
        items = list(items)
        self.entries = (_abi.mrom_packed_obj * len(items))()
        parts, off = [], 0
        for e, it in zip(self.entries, items):
            r = int(it["r"])
            arrs = [np.ascontiguousarray(it["K"], dtype=np.complex128)]
            if it.get("K_in") is not None:
                arrs.append(np.ascontiguousarray(it["K_in"], dtype=np.complex128))
            arrs.append(np.ascontiguousarray(it["C"], dtype=np.complex128))
            if it.get("Me") is not None:
                arrs.append(np.ascontiguousarray(it["Me"], dtype=np.complex128))
            arrs.append(np.ascontiguousarray(it["B"], dtype=np.complex128))
            if it.get("G") is not None:
                arrs.append(np.ascontiguousarray(it["G"], dtype=np.complex128))
            e.r, e.offset = r, off
            e.has_kin, e.has_me, e.has_gram = (int(it.get(k) is not None) for k in ("K_in", "Me", "G"))
            e.c00[:] = [float(v) for v in np.asarray(it["c00"], dtype=np.float64).ravel()]
            e.N0[:] = [float(v) for v in np.asarray(it.get("N0", np.zeros(9)), dtype=np.float64).ravel()]
            e.alpha = float(it.get("alpha", 1.0))
            e.alpha_lb = float(it.get("alpha_lb", 1.0 / np.sqrt(2.0)))
            e.vol_B = float(it.get("vol_B", 1.0))
            for a in arrs:
                parts.append((off, a))
                off += a.nbytes
            off = (off + 15) // 16 * 16
        self.nbytes = off
        host = None
        if pin:
            try:
                import torch
                host = torch.empty(off, dtype=torch.uint8).pin_memory()
                view = host.numpy()
            except Exception:  # no torch / no CUDA for pinning: pageable buffer
                host = None
        if host is None:
            view = np.empty(off, dtype=np.uint8)
            host = view
        for o, a in parts:
            view[o:o + a.nbytes] = a.view(np.uint8).ravel()
        self.buffer = host


def mrom_sweep_host(handle: Handle, packed: PackedDictionary, omega, R, I, Delta=None, n_chunks: int = 2):
    """mrom_sweep_host: the sweep of a PackedDictionary from host memory (omega: n_w float64) into
    host outputs R, I, Delta ([n_obj][n_w][3][3] float64, pinned for overlapped copies; Delta may
    be None), in n_chunks groups pipelined over two streams.  Synchronous."""
    n_w = int(np.asarray(omega.shape)[0]) if hasattr(omega, "shape") else len(omega)
    for x in (omega, R, I, Delta):
        if x is None:
            continue
        if isinstance(x, np.ndarray):
            ok = x.dtype == np.float64
        else:
            ok = x.device.type == "cpu" and str(x.dtype) == "torch.float64"
        if not ok:
            raise ValueError("mrom_sweep_host takes float64 host arrays")
    _abi.check(lib().mrom_sweep_host(handle.ptr, len(packed.entries), packed.entries, _ptr(packed.buffer),
                                     int(packed.nbytes), _ptr(omega), n_w, _ptr(R), _ptr(I), _ptr(Delta),
                                     int(n_chunks)), handle.ptr)


class Plan:
    """mrom_plan: a fixed batch of objects and frequency count (mrom_plan_create)."""

    def __init__(self, handle: Handle, objs, n_w: int):
        self.handle = handle
        self.objs = list(objs)
        self.n_w = int(n_w)
        self._p = ctypes.c_void_p()
        _abi.check(lib().mrom_plan_create(handle.ptr, _rom_array(self.objs), len(self.objs), self.n_w,
                                          ctypes.byref(self._p)), handle.ptr)

    def sweep(self, omega, R, I, Delta=None, omega_stride: int = 0, eig=None):
        """mrom_plan_sweep; with eig (device [n_obj][n_w][6]) mrom_plan_sweep_invariants, which also
        writes the eigenvalues of R~ and I from the sweep's epilogue (R, I may then be None)."""
        if eig is None:
            _abi.check(lib().mrom_plan_sweep(self._p, _ptr(omega), int(omega_stride), _ptr(R), _ptr(I),
                                             _ptr(Delta)), self.handle.ptr)
        else:
            _abi.check(lib().mrom_plan_sweep_invariants(self._p, _ptr(omega), int(omega_stride), _ptr(R), _ptr(I),
                                                        _ptr(Delta), _ptr(eig)), self.handle.ptr)

    def enable_timing(self) -> None:
        """Record CUDA events around the stages of every later sweep (mrom_plan_timing)."""
        _abi.check(lib().mrom_plan_timing(self._p, 1, None), self.handle.ptr)

    def stage_ms(self):
        """(prep, route, pencil sweep, LU sweep) kernel durations of the last sweep, in ms."""
        buf = (ctypes.c_float * 4)()
        _abi.check(lib().mrom_plan_timing(self._p, 0, buf), self.handle.ptr)
        return tuple(float(x) for x in buf)

    def solver_counts(self):
        """(objects on the pencil route, objects on the LU route) of the last sweep."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _abi.check(lib().mrom_plan_solver_counts(self._p, ctypes.byref(a), ctypes.byref(b)), self.handle.ptr)
        return a.value, b.value

    def close(self):
        if self._p:
            lib().mrom_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- C names

def mrom_create(device: int = 0, stream=None) -> Handle:
    return Handle(device, stream)


def mrom_destroy(h: Handle) -> None:
    h.close()


def mrom_synchronize(h: Handle) -> None:
    h.synchronize()


def mrom_last_error(h: Handle) -> str:
    return lib().mrom_last_error(h.ptr).decode()


def mrom_launch_count(h: Handle) -> int:
    return h.launch_count()


def mrom_rom_from_reduced(h: Handle, obj, with_cert: bool = True) -> ReducedObject:
    return ReducedObject.from_workload(h, obj, with_cert=with_cert)


def mrom_rom_free(rom: ReducedObject) -> None:
    rom.close()


def mrom_rom_rank(rom: ReducedObject) -> int:
    return int(lib().mrom_rom_rank(rom.ptr))


def mrom_sweep(h: Handle, objs, omega, n_w: int, R, I, Delta=None, *, omega_stride: int = 0,
               s_sigma=None, s_mu=None) -> None:
    """Device tensors in, device tensors out (R, I, Delta: float64, n_obj*n_w*9)."""
    _abi.check(lib().mrom_sweep(h.ptr, _rom_array(objs), len(objs), _ptr(omega), int(n_w),
                                int(omega_stride), _ptr(s_sigma), _ptr(s_mu), _ptr(R), _ptr(I),
                                _ptr(Delta)), h.ptr)


def mrom_certificate(h: Handle, objs, omega, n_w: int, Delta, *, omega_stride: int = 0) -> None:
    _abi.check(lib().mrom_certificate(h.ptr, _rom_array(objs), len(objs), _ptr(omega), int(n_w),
                                      int(omega_stride), _ptr(Delta)), h.ptr)


def mrom_plan_create(h: Handle, objs, n_w: int) -> Plan:
    return Plan(h, objs, n_w)


def mrom_plan_sweep(plan: Plan, omega, R, I, Delta=None, omega_stride: int = 0) -> None:
    plan.sweep(omega, R, I, Delta, omega_stride)


def mrom_plan_destroy(plan: Plan) -> None:
    plan.close()


def mrom_tune(h: Handle, objs, n_w: int) -> int:
    """Pick the fastest sweep launch configuration for this batch; returns its index."""
    chosen = ctypes.c_int32(-1)
    _abi.check(lib().mrom_tune(h.ptr, _rom_array(objs), len(objs), int(n_w), ctypes.byref(chosen)), h.ptr)
    return int(chosen.value)


def mrom_tune_pencil(h: Handle, objs, n_w: int) -> int:
    """mrom_tune_pencil: picks the pencil sweep's frequency groups per task (8, 4, 2 or 1) by
    timing; returns the choice (the handle's cap for later plans)."""
    chosen = ctypes.c_int32(0)
    _abi.check(lib().mrom_tune_pencil(h.ptr, _rom_array(objs), len(objs), int(n_w), ctypes.byref(chosen)), h.ptr)
    return int(chosen.value)


def mrom_sweep_noalloc(h: Handle, objs, omega, n_w: int, R, I, Delta=None, *, omega_stride: int = 0) -> None:
    """mrom_sweep for callers that cannot allocate device memory while they run.

    Same arguments and results as mrom_sweep (device tensors); all scratch lives in
    a fixed 64 MiB array inside the library.  Calls share that array, so calls
    whose GPU work overlaps must be serialised.
    """
    _abi.check(lib().mrom_sweep_noalloc(h.ptr, _rom_array(objs), len(objs), _ptr(omega), int(n_w),
                                        int(omega_stride), _ptr(R), _ptr(I), _ptr(Delta)), h.ptr)


class FullOrder:
    """Device copy of a full-order problem for mrom_project (torch tensors, caller-owned).

    K: CSR (int32 rowptr, int32 col, float64 val); C, M: lumped diagonals (float64);
    o: (3, n) float64 total theta^(0) coefficients.  The certificate's inner product X is a
    lumped diagonal (X, float64 n) or a sparse SPD matrix (X_csr = (rowptr, col, val) as for K,
    solved by PCG with X_tol and X_max_iter); neither: no certificate.
    """

    def __init__(self, K_rowptr, K_col, K_val, C, o, *, M=None, eps=0.0, X=None, X_csr=None, X_tol=0.0,
                 X_max_iter=0, alpha=1.0, alpha_lb=1.0 / np.sqrt(2.0), vol_B=1.0, N0=None):
        self.keep = [K_rowptr, K_col, K_val, C, o, M, X, N0] + list(X_csr or ())
        f = _abi.mrom_fom()
        f.n = int(C.numel())
        f.K_rowptr, f.K_col, f.K_val = _ptr(K_rowptr), _ptr(K_col), _ptr(K_val)
        f.C_diag, f.M_diag, f.eps = _ptr(C), _ptr(M), float(eps)
        f.o, f.X_diag = _ptr(o), _ptr(X)
        f.alpha, f.alpha_lb, f.vol_B = float(alpha), float(alpha_lb), float(vol_B)
        f.N0 = _ptr(N0)
        if X_csr is not None:
            f.X_rowptr, f.X_col, f.X_val = (_ptr(a) for a in X_csr)
        f.X_tol, f.X_max_iter = float(X_tol), int(X_max_iter)
        self.desc = f
        self.has_cert = X is not None or X_csr is not None

    @classmethod
    def from_fit(cls, problem, device="cuda", *, X=None, alpha_lb=1.0 / np.sqrt(2.0), X_tol=0.0, X_max_iter=0):
        """Upload a workloads.FitProblem (K, C, M, o, eps, alpha, |B|, N0) to the device.  X: the
        certificate's inner product, a diagonal (numpy n) or a scipy sparse SPD matrix, or None."""
        import torch
        K = problem.K.tocsr()
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        X_diag = X_csr = None
        if X is not None and hasattr(X, "tocsr"):
            Xc = X.tocsr()
            Xc.sort_indices()
            X_csr = (t(Xc.indptr, torch.int32), t(Xc.indices, torch.int32), t(Xc.data, torch.float64))
        elif X is not None:
            X_diag = t(X, torch.float64)
        return cls(t(K.indptr, torch.int32), t(K.indices, torch.int32), t(K.data, torch.float64),
                   t(problem.C, torch.float64), t(problem.o, torch.float64), M=t(problem.M, torch.float64),
                   eps=problem.eps, X=X_diag, X_csr=X_csr, X_tol=X_tol, X_max_iter=X_max_iter,
                   alpha=problem.alpha, alpha_lb=alpha_lb, vol_B=problem.vol_B,
                   N0=t(problem.N0.ravel(), torch.float64))


class PermeabilityData:
    """Device copy of the permeability data of a full-order problem (mrom_fom_mu): K_in
    (CSR), x, K x and K_in x (3 x n), the static regularisation's diagonal, the sum over the
    object of |cell| / mu_r, and the static snapshots O (n_o x n float64, one per row)."""

    def __init__(self, Kin_rowptr, Kin_col, Kin_val, x, kx, kx_in, M_static, vol_B_mu, O, *, tol_static=1e-10):
        self.keep = [Kin_rowptr, Kin_col, Kin_val, x, kx, kx_in, M_static, O]
        d = _abi.mrom_fom_mu()
        d.Kin_rowptr, d.Kin_col, d.Kin_val = _ptr(Kin_rowptr), _ptr(Kin_col), _ptr(Kin_val)
        d.x, d.kx, d.kx_in, d.M_static = _ptr(x), _ptr(kx), _ptr(kx_in), _ptr(M_static)
        d.vol_B_mu = float(vol_B_mu)
        d.O, d.ldo, d.n_o = _ptr(O), int(O.shape[1]), int(O.shape[0])
        d.tol_static = float(tol_static)
        self.desc = d

    @classmethod
    def from_fit(cls, problem, O, device="cuda", *, tol_static=1e-10):
        """From a workloads.FitProblem built with mu_split=True and static snapshots O
        (numpy (n_o, n): rows o~_i(s_l))."""
        import torch
        Kin = problem.K_in.tocsr()
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        return cls(t(Kin.indptr, torch.int32), t(Kin.indices, torch.int32), t(Kin.data, torch.float64),
                   t(problem.x, torch.float64), t(problem.kx, torch.float64), t(problem.kx_in, torch.float64),
                   t(problem.eps_static * problem.M_omega, torch.float64), problem.vol_B_mu,
                   t(O, torch.float64), tol_static=tol_static)


def mrom_project_mu(h: Handle, fom: FullOrder, mu: PermeabilityData, D, *, tol_sigma: float = 1e-6,
                    r_max: int = 0):
    """PODP in mu_r: projection onto the basis of the snapshot columns D (device (n_cols, n)
    complex128, taken at sampled (omega, s_mu)) with the reduced static problem of mu.
    Returns (ReducedObject, r, m)."""
    rom = ctypes.c_void_p()
    r_out, m_out = ctypes.c_int32(0), ctypes.c_int32(0)
    _abi.check(lib().mrom_project_mu(h.ptr, ctypes.byref(fom.desc), ctypes.byref(mu.desc), _ptr(D),
                                     int(D.shape[1]), int(D.shape[0]), float(tol_sigma), int(r_max),
                                     ctypes.byref(rom), ctypes.byref(r_out), ctypes.byref(m_out)), h.ptr)
    obj = ReducedObject._wrap(h, rom, r_out.value, fom.has_cert)
    return obj, int(r_out.value), int(m_out.value)


def mrom_rom_mu_state(rom, s_mu: float) -> dict:
    """Reduced static state of an object at s_mu: B, c00, N0 and their derivatives (numpy)."""
    r = rom.r
    out = {k: np.zeros((r, 3), dtype=np.complex128) for k in ("B", "dB")}
    for k in ("c00", "N0", "dc00", "dN0"):
        out[k] = np.zeros(9)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _abi.check(lib().mrom_rom_mu_state(rom.ptr, float(s_mu), out["B"].ctypes.data, dp(out["c00"]), dp(out["N0"]),
                                       out["dB"].ctypes.data, dp(out["dc00"]), dp(out["dN0"])), rom.handle.ptr)
    for k in ("c00", "N0", "dc00", "dN0"):
        out[k] = out[k].reshape(3, 3)
    return out


def mrom_project(h: Handle, fom: FullOrder, D=None, *, tol_sigma: float = 1e-6, r_max: int = 0, basis=None):
    """Off-line stage: TSVD of the snapshot columns D (device (n_cols, n) complex128) and
    projection, or projection onto a given basis (device (n, r) complex128).

    Returns (ReducedObject, singular values (numpy, or None with a basis), rank r).
    """
    rom = ctypes.c_void_p()
    r_out = ctypes.c_int32(0)
    if basis is not None:
        _abi.check(lib().mrom_project(h.ptr, ctypes.byref(fom.desc), None, 0, 0, 0.0, 0, _ptr(basis),
                                      int(basis.shape[1]), ctypes.byref(rom), None, ctypes.byref(r_out)), h.ptr)
        sig = None
    else:
        n_cols = int(D.shape[0])
        sig = np.zeros(n_cols)
        _abi.check(lib().mrom_project(h.ptr, ctypes.byref(fom.desc), _ptr(D), int(D.shape[1]), n_cols,
                                      float(tol_sigma), int(r_max), None, 0, ctypes.byref(rom),
                                      sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.byref(r_out)), h.ptr)
    return ReducedObject._wrap(h, rom, r_out.value, fom.has_cert), sig, int(r_out.value)


def mrom_rom_get(rom: ReducedObject, with_gram: bool = True) -> dict:
    """Host copies of an object's reduced data: K, C, Me, B, c00, G (numpy)."""
    r = rom.r
    out = {k: np.zeros((r, r), dtype=np.complex128) for k in ("K", "C", "Me")}
    out["B"] = np.zeros((r, 3), dtype=np.complex128)
    out["c00"] = np.zeros(9)
    G = np.zeros((2 * r + 3, 2 * r + 3), dtype=np.complex128) if with_gram else None
    _abi.check(lib().mrom_rom_get(rom.ptr, out["K"].ctypes.data, out["C"].ctypes.data, out["Me"].ctypes.data,
                                  out["B"].ctypes.data,
                                  out["c00"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  G.ctypes.data if G is not None else None), rom.handle.ptr)
    out["c00"] = out["c00"].reshape(3, 3)
    out["G"] = G
    return out


def mrom_fom_solve(h: Handle, fom: FullOrder, omegas, *, tol: float = 1e-12, max_iter: int = 100000):
    """Full-order snapshots q_i(omega_k) on the device (COCG, Jacobi preconditioning).
    Returns (Q device (3 n_w, n) complex128 with row 3 k + i = q_i(omega_k), iterations, residuals)."""
    import torch
    w = np.ascontiguousarray(omegas, dtype=np.float64)
    n = int(fom.desc.n)
    Q = torch.empty((3 * w.size, n), dtype=torch.complex128, device="cuda")
    its = np.zeros(3 * w.size, dtype=np.int32)
    res = np.zeros(3 * w.size)
    _abi.check(lib().mrom_fom_solve(h.ptr, ctypes.byref(fom.desc), w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    int(w.size), float(tol), int(max_iter), _ptr(Q), n,
                                    its.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), h.ptr)
    return Q, its, res


def mrom_adapt(h: Handle, fom: FullOrder, omega0, D0, snapshot_fn, omega_out, *, tol_sigma: float = 1e-6,
               tol_delta: float = 1e-3, n_star: int = 2, max_k: int = 10, r_max: int = 0, theta: float = 0.0):
    """Algorithm 1 on the GPU (theta > 0: the variant with a threshold, at most n_star new
    snapshots per iteration).

    omega0: initial snapshot frequencies (numpy); D0: device (3 * ns0, n) complex128
    solution columns; snapshot_fn(omegas) -> numpy (3, n, len(omegas)) full-order
    solutions (called from the library for every refinement), or None: the library solves
    every snapshot itself (mrom_fom_solve) and D0 may be None too; omega_out: device
    float64, strictly increasing.  Returns (ReducedObject, Lambda history, k,
    sorted snapshot frequencies).
    """
    omega0 = np.ascontiguousarray(omega0, dtype=np.float64)
    n = int(fom.desc.n)
    errors = []

    def _cb(user, n_new, omega_ptr, buf):
        try:
            ws = np.ctypeslib.as_array(omega_ptr, shape=(n_new,)).copy()
            D = snapshot_fn(ws)
            dst = np.ctypeslib.as_array(ctypes.cast(buf, ctypes.POINTER(ctypes.c_double)),
                                        shape=(n_new * 3 * n * 2,)).view(np.complex128)
            dst[:] = np.ascontiguousarray(np.transpose(D, (2, 0, 1))).reshape(-1)
            return 0
        except Exception as exc:  # reported as MROM_ECALLBACK
            errors.append(exc)
            return 1

    # a NULL callback (SNAPSHOT_CB()): the library solves the snapshots itself (mrom_fom_solve)
    cb = _abi.SNAPSHOT_CB(_cb) if snapshot_fn is not None else _abi.SNAPSHOT_CB()
    opts = _abi.mrom_adapt_opts(float(tol_sigma), float(tol_delta), int(n_star), int(max_k), int(r_max),
                                  float(theta))
    hist = np.full(max_k, np.nan)
    cap = omega0.size + n_star * max(0, max_k - 1)
    snaps = np.zeros(cap)
    rom = ctypes.c_void_p()
    k = ctypes.c_int32(0)
    ns = ctypes.c_int32(0)
    dp = ctypes.POINTER(ctypes.c_double)
    status = lib().mrom_adapt(h.ptr, ctypes.byref(fom.desc), omega0.ctypes.data_as(dp), omega0.size, _ptr(D0),
                              cb, None, _ptr(omega_out), int(omega_out.numel()), ctypes.byref(opts),
                              ctypes.byref(rom), hist.ctypes.data_as(dp), ctypes.byref(k), snaps.ctypes.data_as(dp),
                              ctypes.byref(ns))
    if errors:
        raise errors[0]
    _abi.check(status, h.ptr)
    obj = ReducedObject._wrap(h, rom, lib().mrom_rom_rank(rom), True)
    return obj, hist[~np.isnan(hist)], int(k.value), snaps[: ns.value]


def mrom_sweep_vjp(h: Handle, objs, omega, n_w: int, gR, gI, g_omega, *, g_ssigma=None, g_smu=None,
                   s_sigma=None, s_mu=None, R=None, I=None, omega_stride: int = 0) -> None:
    """Adjoint of the sweep: dL/domega, dL/ds_sigma, dL/ds_mu for L = <gR, R> + <gI, I> (device tensors)."""
    _abi.check(lib().mrom_sweep_vjp(h.ptr, _rom_array(objs), len(objs), _ptr(omega), int(n_w), int(omega_stride),
                                    _ptr(s_sigma), _ptr(s_mu), _ptr(gR), _ptr(gI), _ptr(g_omega), _ptr(g_ssigma),
                                    _ptr(g_smu), _ptr(R), _ptr(I)), h.ptr)


def mrom_invariants(h: Handle, M, eig) -> None:
    """Eigenvalues (ascending) of the symmetric parts of the 3 x 3 matrices M (device,
    [..., 3, 3]) into eig (device, [..., 3]): the rotation invariants of Sect. 1."""
    n = M.numel() // 9
    if eig.numel() != 3 * n:
        raise ValueError("eig must hold 3 values per 3 x 3 matrix")
    _abi.check(lib().mrom_invariants(h.ptr, _ptr(M), int(n), _ptr(eig)), h.ptr)


def mrom_static_solve(h: Handle, K, M_s, G, GT, f, *, tol: float = 1e-12, max_iter: int = 20000):
    """The regularised static problem (K + M_s) o = f with G^T M_s o = 0.  Device tensors: K, G and
    GT as (rowptr, col, val) CSR triples (int32, int32, float64), M_s (n,) and f (n_rhs, n) float64.
    Returns (o (n_rhs, n) float64 device tensor, iteration counts of the two solves)."""
    import torch
    fom = _abi.mrom_fom()
    fom.n = int(M_s.numel())
    fom.K_rowptr, fom.K_col, fom.K_val = _ptr(K[0]), _ptr(K[1]), _ptr(K[2])
    o = torch.empty_like(f)
    it = (ctypes.c_int32 * 2)()
    _abi.check(lib().mrom_static_solve(h.ptr, ctypes.byref(fom), _ptr(M_s), int(GT[0].numel() - 1),
                                       _ptr(G[0]), _ptr(G[1]), _ptr(G[2]), _ptr(GT[0]), _ptr(GT[1]), _ptr(GT[2]),
                                       _ptr(f), int(f.shape[0]), float(tol), int(max_iter), _ptr(o), it), h.ptr)
    return o, (int(it[0]), int(it[1]))


def static_solver_for(h: Handle, n_grid: int, *, tol: float = 1e-12, device="cuda"):
    """A static_solver(K, M_s, rhs) for workloads.fit_problem on an n_grid^3 FIT grid that runs
    mrom_static_solve (argument marshalling only: uploads K, M_s, the grid's discrete gradient and
    rhs, returns o~ as numpy N x 3)."""
    import torch
    from workloads.fit import node_gradient

    def csr(A):
        A = A.tocsr()
        A.sort_indices()
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)
        return (t(A.indptr, torch.int32), t(A.indices, torch.int32), t(A.data, torch.float64))

    def solve(K, M_s, rhs):
        G = node_gradient(n_grid)
        f = torch.as_tensor(np.ascontiguousarray(np.asarray(rhs).T), dtype=torch.float64, device=device)
        o, its = mrom_static_solve(h, csr(K), torch.as_tensor(M_s, dtype=torch.float64, device=device), csr(G),
                                   csr(G.T), f, tol=tol)
        solve.iters = its
        return o.cpu().numpy().T

    return solve


def mrom_fp64_peak(h: Handle, iters: int = 1 << 16):
    """Measured FP64 pipe throughput of the handle's device: (TFLOP/s, kernel ms)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _abi.check(lib().mrom_fp64_peak(h.ptr, int(iters), ctypes.byref(tf), ctypes.byref(ms)), h.ptr)
    return tf.value, ms.value


def _sweep_values(h, objs, omega, s_sigma, s_mu):
    import torch
    n_obj = len(objs)
    n_w = omega.shape[-1]
    stride = n_w if omega.dim() == 2 else 0
    dev = omega.device
    R = torch.empty((n_obj, n_w, 3, 3), dtype=torch.float64, device=dev)
    I = torch.empty_like(R)
    if s_mu is None:
        mrom_sweep(h, objs, omega.contiguous(), n_w, R, I, omega_stride=stride,
                   s_sigma=None if s_sigma is None else s_sigma.contiguous())
    else:
        z = torch.zeros_like(R)
        g = torch.empty((n_obj, n_w), dtype=torch.float64, device=dev)
        mrom_sweep_vjp(h, objs, omega.contiguous(), n_w, z, z, g, s_sigma=None if s_sigma is None else
                       s_sigma.contiguous(), s_mu=s_mu.contiguous(), R=R, I=I, omega_stride=stride)
    return R, I


def _autograd_function():
    import torch

    class MromSweep(torch.autograd.Function):
        """(omega, s_sigma, s_mu) -> (R, I) with the adjoint kernel as backward."""

        @staticmethod
        def forward(ctx, omega, s_sigma, s_mu, handle, objs):
            R, I = _sweep_values(handle, objs, omega, s_sigma, s_mu)
            ctx.save_for_backward(omega, s_sigma, s_mu)
            ctx.handle, ctx.objs = handle, objs
            return R, I

        @staticmethod
        def backward(ctx, gR, gI):
            omega, s_sigma, s_mu = ctx.saved_tensors
            h, objs = ctx.handle, ctx.objs
            n_obj, n_w = len(objs), omega.shape[-1]
            stride = n_w if omega.dim() == 2 else 0
            dev = omega.device
            gR = torch.zeros((n_obj, n_w, 3, 3), dtype=torch.float64, device=dev) if gR is None else gR.contiguous()
            gI = torch.zeros((n_obj, n_w, 3, 3), dtype=torch.float64, device=dev) if gI is None else gI.contiguous()
            g_w = torch.empty((n_obj, n_w), dtype=torch.float64, device=dev)
            g_ss = torch.empty(n_obj, dtype=torch.float64, device=dev)
            g_sm = torch.empty(n_obj, dtype=torch.float64, device=dev) if s_mu is not None else None
            mrom_sweep_vjp(h, objs, omega.contiguous(), n_w, gR, gI, g_w, g_ssigma=g_ss, g_smu=g_sm,
                           s_sigma=s_sigma, s_mu=s_mu, omega_stride=stride)
            g_omega = g_w if omega.dim() == 2 else g_w.sum(0)
            return (g_omega if ctx.needs_input_grad[0] else None,
                    g_ss if ctx.needs_input_grad[1] else None,
                    g_sm if ctx.needs_input_grad[2] else None, None, None)

    return MromSweep


class _Lazy:
    _fn = None

    def __call__(self):
        if _Lazy._fn is None:
            _Lazy._fn = _autograd_function()
        return _Lazy._fn


MromSweep = _Lazy()


def signature(handle: Handle, objs, omega, s_sigma=None, s_mu=None):
    """Differentiable (R, I) of the objects: omega (n_w,) shared or (n_obj, n_w) per object,
    s_sigma / s_mu (n_obj,) device tensors or None."""
    import torch
    dev = omega.device
    n = len(objs)
    ss = s_sigma if s_sigma is not None else torch.ones(n, dtype=torch.float64, device=dev)
    return MromSweep().apply(omega, ss, s_mu, handle, list(objs))


def mrom_sweep_mixed(h: Handle, objs, omega, n_w: int, R, I, Delta=None, *, n_refine: int = 1,
                     omega_stride: int = 0) -> None:
    """mrom_sweep with complex64 elimination and n_refine float64 refinement steps."""
    _abi.check(lib().mrom_sweep_mixed(h.ptr, _rom_array(objs), len(objs), _ptr(omega), int(n_w),
                                      int(omega_stride), int(n_refine), _ptr(R), _ptr(I), _ptr(Delta)), h.ptr)


def mrom_project_dirs(h: Handle, fom: FullOrder, D=None, *, n_s: int = 0, tol_sigma: float = 1e-6, r_max: int = 0,
                      basis=None, r_dirs=None):
    """One basis per direction (the paper's PODP): D is device (3 * n_s, n) complex128 with the
    snapshots of direction 1, then 2, then 3; or basis (device (n, r1+r2+r3)) with r_dirs.
    Returns (ReducedObject, singular values (3, n_s) or None, (r1, r2, r3))."""
    rom = ctypes.c_void_p()
    rd_out = (ctypes.c_int32 * 3)()
    if basis is not None:
        rd_in = (ctypes.c_int32 * 3)(*[int(x) for x in r_dirs])
        _abi.check(lib().mrom_project_dirs(h.ptr, ctypes.byref(fom.desc), None, 0, 0, 0.0, 0, _ptr(basis), rd_in,
                                           ctypes.byref(rom), None, rd_out), h.ptr)
        sig = None
    else:
        n_s = int(D.shape[0]) // 3
        sig = np.zeros(3 * n_s)
        _abi.check(lib().mrom_project_dirs(h.ptr, ctypes.byref(fom.desc), _ptr(D), int(D.shape[1]), n_s,
                                           float(tol_sigma), int(r_max), None, None, ctypes.byref(rom),
                                           sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), rd_out), h.ptr)
        sig = sig.reshape(3, n_s)
    rd = tuple(int(x) for x in rd_out)
    return ReducedObject._wrap(h, rom, sum(rd), fom.has_cert), sig, rd
