#!/usr/bin/env python
"""Benchmark: spectral-signature tensor evaluations per second on GB300.

Workload (one "step"): the batched dictionary sweep -- 1000 synthetic reduced
objects (shared basis, r drawn uniformly from 8..96, K_r spectrum in
[1e-6, 1e2], C_r spectrum in [1e-3, 1], Gram blocks from a random N = 4096
basis) x 2000 frequencies log-spaced in [1e1, 1e8] rad/s.  Every step runs the
whole on-line path for all 2,000,000 (object, frequency) pairs: reduced solve
(Eq. (17)), R (Eq. (18)), I (Eq. (19)) and the certificate Delta (Lemma 4.2),
in float64: per object the Hermitian-pencil preparation (Cholesky, Householder
tridiagonalisation, implicit QL, transformed Gram blocks), device-side routing,
then the O(r^2)-per-frequency pencil sweep (objects failing the accuracy gate
take the LU sweep in the same step).

value: evaluations/s with the reduced data already resident in HBM.
e2e:   the same through the public API from pinned host buffers -- every step
       uploads the dictionary (mrom_rom_from_reduced_batch), builds the plan,
       sweeps, and reads R, I and Delta back.
roofline: the pencil sweep kernel against the FP64 pipe (GB300: 2 DFMA/clk/SM),
          timed per step with CUDA events around each stage; lu_route: the same
          step with every object on the LU route, for comparison.
cpu_baseline: the CPU oracle (numpy/LAPACK) on a bounded sample of objects.

Multi-GPU (torchrun, N > 1): every rank sweeps its own 1000-object dictionary
(weak scaling, no collective on the data path); value = all evaluations / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spectral-signature tensor evals/sec (objects x freqs), FP64, with certificate"
UNIT = "evals/s"
SM_COUNT_NOMINAL = 152
DFMA_PER_CLK_PER_SM = 2           # GB300 DFMA rate: 4 flop/clk/SM (mrom_fp64_peak measures it in every run)
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one pencil_sweep_kernel launch on
# this workload, from a one-pass ncu capture of the current kernel at full size; None once the kernel
# changes until it is captured again.  The last capture (350.77 MB read + 370.79 MB written) was of
# the kernel before its R and I row sums were regrouped and its frequency groups per task tuned.
SWEEP_DRAM_BYTES_PER_LAUNCH = None
SWEEP_DRAM_NOTE = ("not recaptured since the kernel last changed; the previous version's one-pass "
                   "capture read 350.77 MB and wrote 370.79 MB per launch")
# object groups of the end-to-end leg (mrom_sweep_host)
E2E_CHUNKS = 2


def flops_per_eval(r: int, cert: bool = True) -> float:
    """FP64 flops of one (object, frequency) evaluation as the sweep kernel computes it.

    FMA = 2 flops, multiply = 1; a complex multiply-add is 4 FMA (8 flops).
      form A                      2 FMA per entry                       4 r^2
      elimination, no pivoting    sum_m [m (m+3) updates + m multipliers]
      back substitution           3 right-hand sides
      forms y = (L + D/2) p       3 rhs x r(r+1)/2 per Hermitian matrix (K, C, G~)
      G~(omega) entries           4 FMA per lower-triangle entry
      reductions                  45 length-r dot products
    """
    r = int(r)
    m = np.arange(1, r)
    elim = 8.0 * np.sum(m * (m + 3)) + 6.0 * np.sum(m)
    back = 3 * (8.0 * r * (r - 1) / 2 + 6.0 * r)
    form = 4.0 * r * r
    mats = 3 if cert else 2
    forms = 12.0 * r * (r + 1) * mats + (4.0 * r * (r + 1) if cert else 0.0)
    red = (108.0 + 36.0 + 90.0) * r if cert else (72.0 + 36.0) * r
    return float(elim + back + form + forms + red)


def pencil_sweep_flops(r: int, m_sum: int, n_w: int, cert: bool = True) -> float:
    """FP64 flops of one object's pencil sweep over n_w frequencies (pole-split forms), with
    m_sum = sum over the frequencies of m = #{lambda_k < w}:

      a_k = 1 / (lambda_k + i w) (one division)                 8 per k
      R and I: (lambda den, den) x Re(beta_i^* beta_j)          24 per k
      a_k conj(beta_ki)                                         18 per k
      certificate polynomial Y_kj(w): full suffix (k >= m)      30 per k
        or Horner over five tables (k < m)                      48 per k
      Re(a_k conj(beta_ki) Y_kj), nine (i, j)                    36 per k
      outputs R, I, Delta with the leading-block sums C0(m)     306 per frequency
    """
    r = int(r)
    if not cert:
        return float(n_w * (32 * r + 100))
    return float(n_w * (113 * r + 306) + 18 * m_sum)


def pencil_prep_flops(r: int) -> float:
    """FP64 flops of one object's pencil preparation, counting complex multiply-adds (8 flops):
    Cholesky r^3/6, L^-1 r^3/6, X = L^-1 K r^3/2, H (lower) r^3/6, Householder tridiagonalisation
    r^3, Q1 accumulation 2 r^3/3, V = L^-H Z r^3/2, three transformed Gram blocks 3 x 3 r^3/2
    (the divide-and-conquer eigensolver of the tridiagonal and V = W Q2 are not counted)."""
    r = float(r)
    return 8.0 * r ** 3 * (1 / 6 + 1 / 6 + 1 / 2 + 1 / 6 + 1 + 2 / 3 + 1 / 2 + 4.5) + 8.0 * 9 * r * r


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = os.path.join("/tmp", f"mrom_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, device_index: int = 0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != device_index:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "reasons": sorted(reasons)}


def dictionary(n_obj: int, seed: int):
    from workloads import reduced_dictionary
    return reduced_dictionary(n_obj, seed=seed)


def sample_indices(n_obj: int, n_sample: int) -> np.ndarray:
    """n_sample objects spread evenly over the dictionary (the CPU baseline's and the reference arm's sample)."""
    return np.linspace(0, n_obj - 1, min(n_sample, n_obj)).round().astype(int)


def oracle_sample_rate(objs, omegas, n_sample: int, keep: bool = False):
    """Evaluations/s of the CPU oracle on n_sample objects spread over the dictionary; with keep,
    also its (model, P, R, I, Delta) per sampled object (kept outside the timed loop's arithmetic)."""
    from oracle import certificate, rom
    idx = sample_indices(len(objs), n_sample)
    kept = []
    t0 = time.perf_counter()
    for k in idx:
        model = rom.from_reduced_object(objs[k])
        P = rom.reduced_solve(model, omegas)
        R, I = rom.mm_tensors(model, omegas, P)
        Dl = certificate.certificate(model, omegas, P)
        if keep:
            kept.append((model, P, R, I, Dl))
    dt = time.perf_counter() - t0
    return idx.size * omegas.size / dt, dt, [int(objs[k].r) for k in idx], kept


def accuracy_vs_oracle(omegas, kept, Rg, Ig, Dg) -> dict:
    """Max relative error of the GPU outputs (Rg, Ig, Dg: [n_sample][n_w][3][3], host) against the
    oracle's on the sampled objects at every frequency: R against max_ij |R| per frequency, I and
    Delta against the size of the terms they are sums of (I -> 0 at high omega by cancellation of
    terms of size omega alpha^3/4 |c00|; Delta is a difference of Gram quadratic forms)."""
    from oracle import certificate
    eR = eI = eD = 0.0
    for s, (model, P, R, I, Dl) in enumerate(kept):
        a3 = model.alpha ** 3
        C = model.C[0][0]
        B = np.stack([model.b(i) for i in range(3)], 1)
        absG = np.abs(model.gram)
        Pm = np.stack(P, axis=2)                         # [n_w][r][3]
        hc = np.abs(np.einsum("wki,kl,wlj->wij", Pm.conj(), C, Pm)).reshape(omegas.size, -1).max(1)
        bp = np.abs(np.einsum("ki,wkj->wij", B.conj(), Pm)).reshape(omegas.size, -1).max(1)
        sI = omegas * a3 / 4 * (np.abs(model.c00).max() + hc + 2 * bp)
        sD = np.empty(omegas.size)
        for n, w in enumerate(omegas):
            W = certificate.residual_weights(model, w, [P[i][n] for i in range(3)])
            sD[n] = a3 / (4 * model.alpha_lb) * max(np.abs(x) @ absG @ np.abs(x) for x in W)
        flat = lambda x: x.reshape(omegas.size, -1)
        eR = max(eR, float((np.abs(flat(Rg[s] - R)).max(1) / np.abs(flat(R)).max(1)).max()))
        eI = max(eI, float((np.abs(flat(Ig[s] - I)).max(1) / sI).max()))
        eD = max(eD, float((np.abs(flat(Dg[s] - Dl)).max(1) / sD).max()))
    return {"R": eR, "I": eI, "Delta": eD, "pairs": len(kept) * int(omegas.size),
            "normalisation": "R: |diff| / max_ij |R| per (object, omega); I, Delta: |diff| / term scale"}


def blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        return int(max(n)) if n else os.cpu_count()
    except Exception:
        return os.cpu_count()


def project_flops(n: int, nnz: int, m: int, r: int, cert: bool = True, per_dir: bool = False) -> float:
    """Algorithmic FP64 flops of mrom_project: snapshot Gram (Hermitian half), basis
    apply, SpMM, K_r, C_r, eps M_r (Hermitian half), b, c00 and the certificate Gram.  per_dir
    (mrom_project_dirs): three snapshot Grams of m / 3 columns, each direction's basis from its own."""
    ng = 2 * r + 3
    gram_apply = (3 * 4.0 * n * (m / 3) ** 2 + 8.0 * n * (m / 3) * r) if per_dir else (4.0 * n * m * m + 8.0 * n * m * r)
    fl = gram_apply + 4.0 * nnz * r + 8.0 * n * r * r + 2 * 4.0 * n * r * r
    fl += 8.0 * n * r * 3 + 4.0 * n * 9
    if cert:
        fl += 4.0 * n * ng * ng
    return fl


def measure_projection(m, h, n_grid: int = 96, n_s: int = 32, n_out: int = 10000, snapshots: str = "device"):
    """The 96^3 plain-vs-mixed configuration: a mu_r = 32, sigma = 1.5e6 cube on the n_grid^3 FIT
    grid (N = 2.6M) with the static correction theta~^(0) solved on the device (mrom_static_solve),
    n_s full-order snapshots per direction at log-spaced omega in [1e1, 1e8] solved on the device
    (mrom_fom_solve, Eq. (9)), the paper's PODP with one TSVD per direction (mrom_project_dirs,
    TOL_Sigma 1e-6, r_i <= n_s), projected in float64 and in the mixed mode (complex64 SpMM, Gram
    products on the tensor cores), then n_out outputs of each object (mrom_sweep, float64).  The
    mixed mode's error against the float64 mode per R~ and I entry (R~: |diff| / (max_ij |R~| +
    max_ij |N0|) per frequency, the size of the terms R~ = N0 + R sums; I: |diff| / (omega alpha^3/4
    max |c00|)), and the float64 mode's own projection roofline (FP64 flops)."""
    import torch
    from workloads import CUBE_C2, fit_problem, log_omegas
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if snapshots == "device":
        solver = m.static_solver_for(h, n_grid)
        p = fit_problem(n_grid, CUBE_C2, static_solver=solver)
    else:  # synthetic snapshot columns: the projection alone (no static or full-order solves)
        solver = None
        p = fit_problem(n_grid, CUBE_C2, static=False)
    t_static = time.perf_counter() - t0
    fom = m.FullOrder.from_fit(p)
    ws = log_omegas(1e1, 1e8, n_s)
    per_call = max(1, 48 // 3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = []
    if snapshots == "device":
        Qs = []
        for k in range(0, n_s, per_call):
            Q, it, _ = m.mrom_fom_solve(h, fom, ws[k:k + per_call], tol=1e-12)
            Qs.append(Q)
            its.append(int(it.max()))
        Q = torch.cat(Qs)
        Dd = Q.view(n_s, 3, p.N).transpose(0, 1).reshape(3 * n_s, p.N).contiguous()  # direction-major
        del Q, Qs
    else:
        from workloads.snapshots import synthetic_snapshot_matrix
        Dsyn = synthetic_snapshot_matrix(p.N, n_s, 7, decay=0.42)  # singular values 0.42^k: r = 16 at 1e-6
        Dd = torch.as_tensor(np.ascontiguousarray(Dsyn.transpose(0, 2, 1).reshape(3 * n_s, p.N)), device="cuda")
        del Dsyn
    torch.cuda.synchronize()
    t_fom = time.perf_counter() - t0
    res = {}
    for mixed in (False, True):
        h.set_projection_precision(mixed)
        m.mrom_project_dirs(h, fom, Dd, tol_sigma=1e-6)[0].close()  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rom, _, rd = m.mrom_project_dirs(h, fom, Dd, tol_sigma=1e-6)
        torch.cuda.synchronize()
        res[mixed] = [rom, time.perf_counter() - t0, rd]
    h.set_projection_precision(False)
    wo = log_omegas(1e1, 1e8, n_out)
    om = torch.as_tensor(wo, device="cuda")
    out = {}
    for mixed in (False, True):
        R = torch.empty((1, n_out, 3, 3), dtype=torch.float64, device="cuda")
        I = torch.empty_like(R)
        m.mrom_sweep(h, [res[mixed][0]], om, n_out, R, I)
        h.synchronize()
        t0 = time.perf_counter()
        m.mrom_sweep(h, [res[mixed][0]], om, n_out, R, I)
        h.synchronize()
        out[mixed] = (R[0].cpu().numpy(), I[0].cpu().numpy(), 1e3 * (time.perf_counter() - t0))
    g64 = m.mrom_rom_get(res[False][0], with_gram=False)
    c00 = np.asarray(g64["c00"])
    sR = (np.abs(out[False][0]).reshape(n_out, -1).max(1) + np.abs(p.N0).max())[:, None, None]
    sI = (wo * p.alpha ** 3 / 4 * np.abs(c00).max())[:, None, None]
    eR = (np.abs(out[True][0] - out[False][0]) / sR).max(0)
    eI = (np.abs(out[True][1] - out[False][1]) / sI).max(0)
    rsum = int(sum(res[False][2]))
    fl = project_flops(p.N, p.K.nnz, 3 * n_s, rsum, cert=False, per_dir=True)
    dt = res[False][1]
    for mixed in (False, True):
        res[mixed][0].close()
    desc = (f"{n_s} device-solved snapshots per direction in [1e1, 1e8]" if snapshots == "device" else
            f"{n_s} synthetic snapshot columns per direction (singular values 0.42^k)")
    return {"workload": f"{n_grid}^3 FIT grid (N = {p.N}, {p.K.nnz} nnz), mu_r = 32 cube"
                        + (" with the static correction, " if snapshots == "device" else ", ")
                        + f"{desc}, one TSVD per direction (TOL_Sigma 1e-6 -> r = {list(res[False][2])}), "
                        f"{n_out} outputs",
            "static_solve_seconds_with_assembly": t_static,
            "static_iterations": list(solver.iters) if solver is not None else None,
            "snapshot_solve_seconds": t_fom, "snapshot_iterations_max": its,
            "project_seconds": {"fp64": dt, "mixed": res[True][1]}, "r_dirs_mixed": list(res[True][2]),
            "sweep_ms": {"fp64": out[False][2], "mixed": out[True][2]},
            "fp64_project_flops": fl, "fp64_project_frac": fl / dt / 1e12 / (SM_COUNT_NOMINAL * DFMA_PER_CLK_PER_SM * 2 * 2.07e9 / 1e12),
            "mixed_vs_fp64_per_entry": {"R": eR.round(12).tolist(), "I": eI.round(12).tolist(),
                                        "max_R": float(eR.max()), "max_I": float(eI.max()),
                                        "normalisation": "R~: |diff| / (max|R~| + max|N0|); I: |diff| / "
                                                         "(omega alpha^3/4 max|c00|), per frequency"}}


def measure_podp_mu(m, h, stream, n_grid=16, n_inst=1000, n_w=2000):
    """PODP in mu_r: a magnetic cube (mu_r = 16 at s = 1) projected once from full-order snapshots
    (solved on the device by mrom_fom_solve) at 3 permeability scales x 4 frequencies
    (mrom_project_mu), then n_inst instances at
    s_mu log-uniform in [1/4, 4] and s_sigma = 1 over n_w frequencies in [1e1, 1e6], values and
    the permeability gradient (mrom_sweep_vjp, B, c00 and N0 following s_mu).  Accuracy: two
    instances between the samples against full-order solves (the method's error, not parity)."""
    import torch
    from oracle import fom as ofom
    from workloads import fit_problem, log_omegas
    from workloads.fit import Material
    mat = (Material((0.375,) * 3, (0.625,) * 3, 5.96e6, 16.0),)
    S = (0.25, 1.0, 4.0)  # sampled permeability scales
    Ws = log_omegas(1e1, 1e6, 4)
    probs = {s: fit_problem(n_grid, mat, mu_scale=s, mu_split=True) for s in S}
    # dynamic snapshots by the device solver (mrom_fom_solve), one call per sampled scale
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dcols = torch.cat([m.mrom_fom_solve(h, m.FullOrder.from_fit(probs[s]), Ws, tol=1e-12)[0] for s in S], dim=0)
    torch.cuda.synchronize()
    t_fom = time.perf_counter() - t0
    p1 = probs[1.0]
    O = np.concatenate([probs[s].o_tilde for s in S], axis=0)
    fom = m.FullOrder.from_fit(p1, X=p1.eps * p1.M + 1e1 * p1.C)  # certificate inner product, omega_min = 10
    mu = m.PermeabilityData.from_fit(p1, O, tol_static=1e-8)
    m.mrom_project_mu(h, fom, mu, dcols, tol_sigma=1e-8)[0].close()  # warm-up
    t0 = time.perf_counter()
    rom, r, mm = m.mrom_project_mu(h, fom, mu, dcols, tol_sigma=1e-8)
    t_proj = time.perf_counter() - t0
    rng = np.random.default_rng(20230714)
    s_mu = np.exp(rng.uniform(np.log(0.25), np.log(4.0), n_inst))
    s_mu[:2] = (0.5, 2.0)
    wo = log_omegas(1e1, 1e6, n_w)
    dev = torch.device("cuda")
    om = torch.as_tensor(wo, device=dev)
    sm = torch.as_tensor(s_mu, device=dev)
    shape = (n_inst, n_w, 3, 3)
    gR = torch.as_tensor(rng.standard_normal(shape), device=dev)
    gI = torch.as_tensor(rng.standard_normal(shape), device=dev)
    R = torch.empty(shape, dtype=torch.float64, device=dev)
    I = torch.empty_like(R)
    g_w = torch.empty((n_inst, n_w), dtype=torch.float64, device=dev)
    g_m = torch.empty(n_inst, dtype=torch.float64, device=dev)
    objs = [rom] * n_inst

    def step():
        m.mrom_sweep_vjp(h, objs, om, n_w, gR, gI, g_w, g_smu=g_m, s_mu=sm, R=R, I=I)

    step()
    h.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        step()
    e1.record(stream)
    h.synchronize()
    ms = e0.elapsed_time(e1) / 3
    # values and the certificate at each instance's scale (mrom_sweep with s_mu and Delta)
    Dl = torch.empty_like(R)

    def cert_step():
        m.mrom_sweep(h, objs, om, n_w, R, I, Dl, s_mu=sm)

    cert_step()
    h.synchronize()
    e0.record(stream)
    for _ in range(3):
        cert_step()
    e1.record(stream)
    h.synchronize()
    ms_cert = e0.elapsed_time(e1) / 3
    dmax_mid = float(Dl[:, n_w // 2].abs().max().item())
    # the method's error between the samples: full-order solves at s = 0.5 and 2 on a few frequencies
    idx = np.array([0, n_w // 3, 2 * n_w // 3, n_w - 1])
    err = []
    for k, s in enumerate((0.5, 2.0)):
        p = fit_problem(n_grid, mat, mu_scale=s)
        Rf, If = ofom.fmm_signature(p, wo[idx])
        Rf = Rf + p.N0[None]
        Rg, Ig = R[k, idx].cpu().numpy(), I[k, idx].cpu().numpy()
        o = p.x + p.o_tilde
        sI = wo[idx] * p.alpha ** 3 / 4 * np.abs(o @ (p.C[:, None] * o.T)).max()
        eR = np.abs(Rg - Rf).reshape(idx.size, -1).max(1) / np.abs(Rf).reshape(idx.size, -1).max(1)
        eI = np.abs(Ig - If).reshape(idx.size, -1).max(1) / sI
        err.append(float(max(eR.max(), eI.max())))
    rom.close()
    return {"workload": f"PODP in mu_r: {n_grid}^3 FIT cube (N = {p1.N}), mu_r = 16 x s, sigma = 5.96e6; "
                        f"snapshots at s in {list(S)} x 4 omega in [1e1, 1e6]; {n_inst} instances with s_mu "
                        f"log-uniform in [1/4, 4] x {n_w} omega in [1e1, 1e6], values and dL/ds_mu",
            "r": r, "m_static": mm, "project_seconds": t_proj, "full_order_snapshot_seconds_device": t_fom,
            "ms_per_step": ms, "value": n_inst * n_w / (ms * 1e-3),
            "unit": "(s_mu, omega) evaluations/s with the permeability gradient",
            "with_certificate": {"ms_per_step": ms_cert, "value": n_inst * n_w / (ms_cert * 1e-3),
                                 "unit": "(s_mu, omega) evaluations/s of R, I and Delta at each instance's scale",
                                 "max_delta_mid_frequency": dmax_mid},
            "max_rel_error_vs_full_order_between_samples": max(err)}


def measure_c1_latency(m, h):
    """Copper cube on the 16^3 FIT grid (N = 10,800): the paper's PODP with one TSVD per direction
    from nine full-order snapshots in [1e1, 1e5] (computed on the host by sparse LU: the off-line
    inputs), then 100 outputs with the certificate.  Wall time of project + sweep (latency)."""
    import torch
    from workloads import CUBE_C1, fit_problem, full_order_snapshots, log_omegas
    p = fit_problem(16, CUBE_C1)
    D = full_order_snapshots(p, log_omegas(1e1, 1e5, 9))
    X = p.eps * p.M + 10.0 * p.C
    fom = m.FullOrder.from_fit(p, X=X)
    cols = torch.as_tensor(np.ascontiguousarray(np.concatenate([D[i].T for i in range(3)])), device="cuda")
    om = torch.as_tensor(log_omegas(1e1, 1e5, 100), device="cuda")
    R = torch.empty((1, 100, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    Dl = torch.empty_like(R)
    times = []
    for _ in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        obj, _, rd = m.mrom_project_dirs(h, fom, cols, tol_sigma=1e-6)
        t1 = time.perf_counter()
        m.mrom_sweep(h, [obj], om, 100, R, I, Dl)
        h.synchronize()
        t2 = time.perf_counter()
        obj.close()
        times.append((t1 - t0, t2 - t1))
    tp, ts = np.median(np.array(times[1:]), axis=0)
    return {"workload": "c1: 16^3 copper cube (N = 10800), 9 snapshots in [1e1, 1e5], one TSVD per direction, "
                        "100 outputs with certificate", "r_dirs": list(rd), "project_ms": 1e3 * tp,
            "sweep_ms": 1e3 * ts, "total_ms": 1e3 * (tp + ts)}


def measure_fom_solve(m, h, n_grid: int = 128, n_w: int = 2):
    """mrom_fom_solve alone: the 3 n_w right-hand sides of n_w frequencies (log-spaced in
    [1e1, 1e8]) on the n_grid^3 two-material grid, Jacobi-scaled residual 1e-12; per-iteration
    rates from the iteration counts (the CSR K is read once per iteration for all columns)."""
    import torch
    from workloads import TWO_MATERIAL_C5, fit_problem, log_omegas
    p = fit_problem(n_grid, TWO_MATERIAL_C5, static=False)
    fom = m.FullOrder.from_fit(p)
    ws = log_omegas(1e1, 1e8, n_w)
    m.mrom_fom_solve(h, fom, ws[:1], tol=1e-6)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Q, its, res = m.mrom_fom_solve(h, fom, ws, tol=1e-12)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    nit = int(its.max())
    nnz = int(p.K.nnz)
    nc = 3 * n_w
    flops = nit * nc * (4.0 * nnz + 40.0 * p.N)   # SpMV 4 per nonzero, ~40 per row in the vector kernels
    return {"workload": f"mrom_fom_solve: {n_grid}^3 two-material FIT grid (N = {p.N}, nnz(K) = {nnz}), "
                        f"{nc} right-hand sides at {n_w} frequencies in [1e1, 1e8]",
            "seconds": sec, "iterations_max": nit, "iterations_min": int(its.min()),
            "ms_per_iteration": sec * 1e3 / nit, "ms_per_column_iteration": sec * 1e3 / nit / nc,
            "approx_fp64_tflops": flops / sec / 1e12, "scaled_residual_max": float(res.max())}


def measure_adaptive_fom(m, h, n_grid: int = 128, ns0: int = 9, n_star: int = 2, max_k: int = 28,
                         n_out: int = 4096, cert_x: str = "sparse"):
    """Algorithm 1 end to end on the device: mrom_adapt without a callback, so every full-order
    snapshot of Eq. (9) is solved by mrom_fom_solve (COCG, Jacobi-scaled residual 1e-12), on the
    n_grid^3 two-material grid with the static correction theta~^(0) of the mu_r = 64 cube solved
    on the device (mrom_static_solve), 4096 outputs in [1e1, 1e8], shared basis, r <= 64, and the
    certificate in the inner product X = K + eps M + omega_min C (sparse, PCG on the device;
    cert_x "diag": X = eps M + omega_min C).  Also times one batched solve of the 3 x 9 initial
    right-hand sides."""
    import torch
    from workloads import TWO_MATERIAL_C5, fit_problem, log_omegas
    import scipy.sparse as sp
    t0 = time.perf_counter()
    solver = m.static_solver_for(h, n_grid)
    p = fit_problem(n_grid, TWO_MATERIAL_C5, static_solver=solver)
    t_static = time.perf_counter() - t0
    wo = log_omegas(1e1, 1e8, n_out)
    Xd = p.eps * p.M + wo[0] * p.C
    X = (p.K + sp.diags(Xd)).tocsr() if cert_x == "sparse" else Xd
    fom = m.FullOrder.from_fit(p, X=X)
    w0 = log_omegas(1e1, 1e8, ns0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Q, its, res = m.mrom_fom_solve(h, fom, w0, tol=1e-12)
    t_solve = time.perf_counter() - t0
    del Q
    om = torch.as_tensor(wo, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rom, hist, k, snaps = m.mrom_adapt(h, fom, w0, None, None, om, tol_sigma=1e-6, tol_delta=1e-3,
                                       n_star=n_star, max_k=max_k, r_max=64)
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    r = rom.r
    rom.close()
    lam = hist[~np.isnan(hist)]
    b_alpha = p.alpha ** 3 * p.vol_B
    return {"workload": f"mrom_adapt with device snapshots: {n_grid}^3 two-material FIT grid (N = {p.N}), "
                        f"static theta~^(0) by mrom_static_solve, {ns0} -> {len(snaps)} snapshots (+{n_star} per "
                        f"iteration), {n_out} output frequencies, shared basis, r_max 64, certificate inner product "
                        f"{'K + eps M + omega_min C (sparse)' if cert_x == 'sparse' else 'eps M + omega_min C'}",
            "iterations": int(k), "final_r": int(r), "seconds_total": total,
            "seconds_per_iteration": total / max(1, k - 1),
            "lambda_over_B_history": [float(x) / b_alpha for x in lam],
            "lambda_over_B_last": float(lam[-1]) / b_alpha if lam.size else None,
            "reached_tol_delta": bool(lam.size and lam[-1] / b_alpha <= 1e-3),
            "static_solve": {"seconds_with_assembly": t_static, "iterations": list(solver.iters)},
            "initial_solve": {"rhs": 3 * ns0, "seconds": t_solve, "iterations_max": int(its.max()),
                              "iterations_min": int(its.min()), "scaled_residual_max": float(res.max())}}


def measure_adaptive(m, h, n_grid: int = 128, ns0: int = 9, n_star: int = 2, max_k: int = 28, n_out: int = 4096):
    """Algorithm 1 (mrom_adapt) on the n_grid^3 two-material FIT grid (128^3: N = 6.2M) with
    4096 output frequencies in [1e1, 1e8], shared basis, r <= 64.  The full-order solves are out
    of reach here, so the snapshot callback returns synthetic columns instead: fixed random
    patterns per direction (on the GPU) combined with geometrically decaying random weights.  The
    record separates the callback's time from the library's (certificates on the output grid,
    interval maxima, TSVD and re-projection)."""
    import torch
    from workloads import TWO_MATERIAL_C5, fit_problem, log_omegas
    p = fit_problem(n_grid, TWO_MATERIAL_C5, static=False)
    wo = log_omegas(1e1, 1e8, n_out)
    X = p.eps * p.M + wo[0] * p.C
    fom = m.FullOrder.from_fit(p, X=X)
    g = torch.Generator(device="cuda")
    g.manual_seed(20230714)
    K = 32
    P = [torch.complex(torch.randn(p.N, K, generator=g, device="cuda", dtype=torch.float64),
                       torch.randn(p.N, K, generator=g, device="cuda", dtype=torch.float64)) / np.sqrt(2 * p.N)
         for _ in range(3)]
    decay = torch.as_tensor(0.55 ** np.arange(K), device="cuda").to(torch.complex128)
    cb_time = [0.0]

    def columns(ws):  # (3, N, len(ws)) on the device
        c = torch.complex(torch.randn(3, K, len(ws), generator=g, device="cuda", dtype=torch.float64),
                          torch.randn(3, K, len(ws), generator=g, device="cuda", dtype=torch.float64))
        return torch.stack([P[i] @ (decay[:, None] * c[i]) for i in range(3)])

    def snapshot_fn(ws):
        t0 = time.perf_counter()
        out = columns(ws).cpu().numpy()
        cb_time[0] += time.perf_counter() - t0
        return out

    w0 = log_omegas(1e1, 1e8, ns0)
    D0 = columns(w0).permute(2, 0, 1).reshape(3 * ns0, p.N).contiguous()
    om = torch.as_tensor(wo, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rom, hist, k, snaps = m.mrom_adapt(h, fom, w0, D0, snapshot_fn, om, tol_sigma=1e-6, tol_delta=1e-3,
                                       n_star=n_star, max_k=max_k, r_max=64)
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    r = rom.r
    rom.close()
    return {"workload": f"mrom_adapt: {n_grid}^3 two-material FIT grid (N = {p.N}), {ns0} -> {len(snaps)} snapshots "
                        f"(+{n_star} per iteration), {n_out} output frequencies, shared basis, r_max 64; synthetic "
                        f"snapshot columns from the callback",
            "iterations": int(k), "final_r": int(r), "seconds_total": total, "seconds_callback": cb_time[0],
            "seconds_library": total - cb_time[0], "seconds_per_iteration": (total - cb_time[0]) / max(1, k - 1),
            "lambda_last": float(hist[~np.isnan(hist)][-1]) if np.any(~np.isnan(hist)) else None}


def config(args):
    return {"workload": f"batched dictionary sweep: {args.n_obj} reduced objects (r ~ U{{8..96}}, shared basis) "
                        f"x {args.n_w} log-spaced omega in [1e1, 1e8] rad/s; R, I and certificate Delta",
            "n_obj": args.n_obj, "n_w": args.n_w, "r_range": [8, 96], "omega_range": [1e1, 1e8],
            "certificate": True, "precision": "fp64",
            "l2": "inputs larger than L2: 0.39 GB reduced data read and 0.43 GB written per step"}


def run_reference(args, world):
    """The oracle as it stands, timed on the host cores (bounded sample per step)."""
    from workloads import log_omegas
    objs = dictionary(args.n_obj, 20230711)
    wo = log_omegas(1e1, 1e8, args.n_w)
    n_s = min(args.ref_sample, len(objs))
    for _ in range(args.warmup):
        oracle_sample_rate(objs, wo, 1)
    times = []
    for _ in range(args.steps):
        rate, dt, rs, _ = oracle_sample_rate(objs, wo, n_s)
        times.append(dt)
    evals = n_s * args.n_w
    value = evals * len(times) / sum(times)
    cores = blas_threads()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_s} objects spread over the dictionary (r = {rs}, mean {np.mean(rs):.1f}) "
                                   f"x {args.n_w} frequencies per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)  # about 0.8 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-obj", type=int, default=1000)
    ap.add_argument("--n-w", type=int, default=2000)
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--e2e-chunks", type=int, default=E2E_CHUNKS,
                    help="object groups of the end-to-end leg (mrom_sweep_host n_chunks)")
    ap.add_argument("--cpu-sample", type=int, default=20)
    ap.add_argument("--ref-sample", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--lu-route", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--gradients", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: every rank its own dictionary (weak) or one dictionary split by cost (strong)")
    ap.add_argument("--projection-only", action="store_true",
                    help="time mrom_project alone (float64 and complex64 products) and print its record")
    ap.add_argument("--projection-grid", type=int, default=96)
    ap.add_argument("--projection-snapshots", default="device", choices=["device", "synthetic"],
                    help="snapshot columns of the projection section: solved on the device, or synthetic")
    ap.add_argument("--adaptive-only", action="store_true",
                    help="time mrom_adapt (Algorithm 1) on the two-material grid and print its record")
    ap.add_argument("--adaptive-grid", type=int, default=128)
    ap.add_argument("--fom-solve-only", action="store_true", help="time mrom_fom_solve alone and print its record")
    ap.add_argument("--fom-grid", type=int, default=128)
    ap.add_argument("--fom-freqs", type=int, default=2)
    ap.add_argument("--adaptive-fom", action="store_true",
                    help="with --adaptive-only: solve the full-order snapshots on the device (no callback)")
    ap.add_argument("--cert-x", default="sparse", choices=["sparse", "diag"],
                    help="--adaptive-fom: certificate inner product K + eps M + omega_min C, or its diagonal part")
    ap.add_argument("--adaptive-max-k", type=int, default=28)
    ap.add_argument("--projection", action=argparse.BooleanOptionalAction, default=True)
    ap.add_argument("--podp-mu", action=argparse.BooleanOptionalAction, default=True,
                    help="PODP in mu_r section (projection with the static reduction, instances over s_mu)")
    ap.add_argument("--podp-mu-only", action="store_true", help="run only the PODP in mu_r section")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, world)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    import paper_2307_05590_gb300 as m
    from workloads import log_omegas

    if args.adaptive_only:
        stream = torch.cuda.Stream(dev)
        h = m.Handle(local_rank, stream.cuda_stream)
        if rank == 0:
            if args.adaptive_fom:
                rec = measure_adaptive_fom(m, h, n_grid=args.adaptive_grid, cert_x=args.cert_x,
                                           max_k=args.adaptive_max_k)
            else:
                rec = measure_adaptive(m, h, n_grid=args.adaptive_grid)
            print(json.dumps({"adaptive": rec}), flush=True)
        h.close()
        return

    if args.fom_solve_only:
        stream = torch.cuda.Stream(dev)
        h = m.Handle(local_rank, stream.cuda_stream)
        if rank == 0:
            print(json.dumps({"fom_solve": measure_fom_solve(m, h, n_grid=args.fom_grid, n_w=args.fom_freqs)}),
                  flush=True)
        h.close()
        return

    if args.podp_mu_only:
        stream = torch.cuda.Stream(dev)
        h = m.Handle(local_rank, stream.cuda_stream)
        with torch.cuda.stream(stream):
            if rank == 0:
                print(json.dumps({"podp_mu": measure_podp_mu(m, h, stream)}), flush=True)
        h.close()
        return

    if args.projection_only:
        stream = torch.cuda.Stream(dev)
        h = m.Handle(local_rank, stream.cuda_stream)
        if rank == 0:
            print(json.dumps({"projection": measure_projection(m, h, n_grid=args.projection_grid,
                                                               snapshots=args.projection_snapshots)}), flush=True)
        h.close()
        return

    from paper_2307_05590_gb300 import shard
    if args.scaling == "weak" or world == 1:
        objs = dictionary(args.n_obj, 20230711 + rank)   # every rank its own dictionary
    else:                                                 # one dictionary split by cost
        full = dictionary(args.n_obj, 20230711)
        part = shard.balanced_split(shard.sweep_cost([o.r for o in full], args.n_w), world)[rank]
        objs = [full[k] for k in part]
        args.n_obj = len(objs)
    wo = log_omegas(1e1, 1e8, args.n_w)
    rs = np.array([o.r for o in objs])
    flops_lu = float(sum(flops_per_eval(r) for r in rs)) * args.n_w
    # m = #{lambda_k < omega} per object and frequency (host eigenvalues of the pencil (K, C))
    m_sums = [int(np.searchsorted(np.sort(sla.eigh(o.K, o.C, eigvals_only=True)), wo).sum()) for o in objs]
    flops_pen = float(sum(pencil_sweep_flops(r, ms, args.n_w) for r, ms in zip(rs, m_sums)))
    flops_prep = float(sum(pencil_prep_flops(r) for r in rs))

    stream = torch.cuda.Stream(dev)
    h = m.Handle(local_rank, stream.cuda_stream)
    roms = [m.ReducedObject.from_workload(h, o) for o in objs]
    sweep_cfg = m.mrom_tune(h, roms, args.n_w)
    pencil_groups = m.mrom_tune_pencil(h, roms, args.n_w)
    plan = m.Plan(h, roms, args.n_w)
    plan.enable_timing()
    om = torch.as_tensor(wo, dtype=torch.float64, device=dev)
    shape = (args.n_obj, args.n_w, 3, 3)
    R = torch.empty(shape, dtype=torch.float64, device=dev)
    I = torch.empty_like(R)
    D = torch.empty_like(R)

    for _ in range(args.warmup):
        plan.sweep(om, R, I, D)
    h.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stages = []
    n0 = h.launch_count()
    t0 = time.perf_counter()
    for k in range(args.steps):
        ev[k][0].record(stream)
        plan.sweep(om, R, I, D)
        ev[k][1].record(stream)
        stages.append(plan.stage_ms())  # (prep, route, pencil sweep, LU sweep) of this step
    h.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = h.launch_count() - n0
    clk = clocks.stop(local_rank)
    per_launch_ms = [a.elapsed_time(b) for a, b in ev]
    dev_ms = ev[0][0].elapsed_time(ev[-1][1])
    ms_per_step = shard.max_over_ranks(dev_ms / args.steps, device=dev)   # the slowest rank
    evals_step = int(shard.sum_over_ranks(args.n_obj * args.n_w, device=dev))
    value = evals_step / (ms_per_step * 1e-3)

    n_pen, n_lu = plan.solver_counts()
    # the sampled objects' outputs of the last timed step, for the accuracy check against the oracle
    acc_idx = torch.as_tensor(sample_indices(args.n_obj, args.cpu_sample), device=dev)
    acc_out = [x.index_select(0, acc_idx).cpu().numpy() for x in (R, I, D)]

    # ---- end to end through the public API from pinned host buffers
    # (measured right after the timed device steps, in the same thermal and clock state; the later
    # sections run seconds of full FP64 load that slow any step measured after them)
    e2e = None
    if args.e2e_steps > 0:
        # the dictionary in one pinned host buffer (mrom_rom_from_packed copies it in one transfer)
        packed = m.PackedDictionary([dict(r=o.r, K=o.K, C=o.C, B=o.B, c00=o.c00, G=o.G, K_in=o.K_in,
                                          alpha=o.alpha, alpha_lb=o.alpha_lb, vol_B=o.vol_B) for o in objs])
        h2d = packed.nbytes + 72 * len(objs)
        om_host = torch.from_numpy(wo.copy()).pin_memory()
        h2d += om_host.numel() * 8
        outs = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(3)]
        d2h = 3 * int(np.prod(shape)) * 8

        def e2e_step():
            # host buffers in and out; the library pipelines upload, sweep and read-back by groups
            m.mrom_sweep_host(h, packed, om_host, outs[0], outs[1], outs[2], n_chunks=args.e2e_chunks)

        with torch.cuda.stream(stream):
            e2e_step()
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                e2e_step()
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            te = torch.tensor([(time.perf_counter() - t0) / args.e2e_steps], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": evals_step / float(te.item()), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * float(te.item()),
               "api": f"mrom_sweep_host, {args.e2e_chunks} object groups pipelined over two streams"}

    # ---- rotation invariants (eigenvalues of R~ and I per frequency) of the step's outputs
    eigs = torch.empty((args.n_obj, args.n_w, 3), dtype=torch.float64, device=dev)
    m.mrom_invariants(h, R, eigs)
    h.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    m.mrom_invariants(h, R, eigs)
    m.mrom_invariants(h, I, eigs)
    e1.record(stream)
    h.synchronize()
    ms_inv = e0.elapsed_time(e1)
    del eigs
    # the same invariants fused into the sweep's epilogue (mrom_plan_sweep_invariants): the step's
    # extra time over the plain step
    E6 = torch.empty((args.n_obj, args.n_w, 6), dtype=torch.float64, device=dev)
    plan.sweep(om, R, I, D, eig=E6)
    h.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        plan.sweep(om, R, I, D, eig=E6)
    e1.record(stream)
    h.synchronize()
    ms_fused = e0.elapsed_time(e1) / args.steps
    del E6
    inv = {"standalone_ms_for_R_and_I": ms_inv, "matrices": 2 * args.n_obj * args.n_w,
           "fused_step_ms": ms_fused, "fused_extra_ms": ms_fused - ms_per_step,
           "method": "closed form (trigonometric outermost eigenvalue, deflation, 2 x 2), FP64"}

    # ---- the same step with every object on the LU route (float64 elimination)
    lu_route = None
    if args.lu_route:
        h.set_solver(lu=True)
        plan_lu = m.Plan(h, roms, args.n_w)
        R2, I2, D2 = torch.empty_like(R), torch.empty_like(R), torch.empty_like(R)
        plan_lu.sweep(om, R2, I2, D2)
        h.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            plan_lu.sweep(om, R2, I2, D2)
        e1.record(stream)
        h.synchronize()
        ms_lu = e0.elapsed_time(e1) / 2

        def rel_d(a, b):
            sc = torch.clamp(b.abs().amax(dim=(2, 3), keepdim=True), min=1e-300)
            return float(((a - b).abs() / sc).max().item())
        lu_route = {"value": args.n_obj * args.n_w / (ms_lu * 1e-3), "unit": UNIT, "ms_per_step": ms_lu,
                    "achieved_tflops": flops_lu / (ms_lu * 1e-3) / 1e12,
                    "max_rel_diff_vs_pencil": {"R": rel_d(R2, R), "I": rel_d(I2, I), "Delta": rel_d(D2, D)}}
        plan_lu.close()
        h.set_solver(lu=False)
        del R2, I2, D2

    # ---- mixed precision (complex64 elimination + one float64 refinement step), same dictionary
    mixed = None
    if args.mixed:
        Rm, Im, Dm = torch.empty_like(R), torch.empty_like(R), torch.empty_like(R)
        for _ in range(2):
            m.mrom_sweep_mixed(h, roms, om, args.n_w, Rm, Im, Dm, n_refine=1)
        h.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_mixed = min(args.steps, 3)  # about 1.3 s per step
        e0.record(stream)
        for _ in range(n_mixed):
            m.mrom_sweep_mixed(h, roms, om, args.n_w, Rm, Im, Dm, n_refine=1)
        e1.record(stream)
        h.synchronize()
        ms_mixed = e0.elapsed_time(e1) / n_mixed
        # error against the float64 sweep, normwise per tensor (R: max|R|, I and Delta: max of both)
        def rel(a, b):
            sc = torch.clamp(b.abs().amax(dim=(2, 3), keepdim=True), min=1e-300)
            return float(((a - b).abs() / sc).max().item())
        def rel_entries(a, b):  # per (i, j): max over objects and frequencies, same normalisation
            sc = torch.clamp(b.abs().amax(dim=(2, 3), keepdim=True), min=1e-300)
            return ((a - b).abs() / sc).amax(dim=(0, 1)).cpu().numpy().round(15).tolist()
        mixed = {"value": args.n_obj * args.n_w / (ms_mixed * 1e-3), "unit": UNIT, "ms_per_step": ms_mixed,
                 "n_refine": 1, "max_rel_err_vs_fp64": {"R": rel(Rm, R), "I": rel(Im, I), "Delta": rel(Dm, D)},
                 "max_rel_err_per_entry": {"R": rel_entries(Rm, R), "I": rel_entries(Im, I)},
                 "normalisation": "|difference| / max_ij |FP64 value| at the same object and frequency"}
        del Rm, Im, Dm

    proj = measure_projection(m, h) if args.projection else None
    pmu = measure_podp_mu(m, h, stream) if args.podp_mu and rank == 0 else None
    c1 = measure_c1_latency(m, h) if args.projection else None

    # ---- gradients (adjoint sweep) on the same dictionary: dL/domega, dL/ds_sigma, dL/ds_mu for
    # per-object scales s_sigma ~ U(0.5, 2), s_mu ~ U(1, 64) and random cotangents of R and I
    grads = None
    if args.gradients:
        rng = np.random.default_rng(20230713)
        ss = torch.as_tensor(rng.uniform(0.5, 2.0, args.n_obj), device=dev)
        sm = torch.as_tensor(rng.uniform(1.0, 64.0, args.n_obj), device=dev)
        gR = torch.as_tensor(rng.standard_normal(shape), device=dev)
        gI = torch.as_tensor(rng.standard_normal(shape), device=dev)
        g_w = torch.empty((args.n_obj, args.n_w), dtype=torch.float64, device=dev)
        g_s = torch.empty(args.n_obj, dtype=torch.float64, device=dev)
        g_m = torch.empty_like(g_s)

        def vjp():
            m.mrom_sweep_vjp(h, roms, om, args.n_w, gR, gI, g_w, g_ssigma=g_s, g_smu=g_m, s_sigma=ss, s_mu=sm,
                             R=R, I=I)
        vjp()
        h.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            vjp()
        e1.record(stream)
        h.synchronize()
        ms_vjp = e0.elapsed_time(e1) / 2
        grads = {"value": args.n_obj * args.n_w / (ms_vjp * 1e-3), "unit": "gradient evals/s (R, I and their "
                 "vector-Jacobian product w.r.t. omega, s_sigma, s_mu)", "ms_per_step": ms_vjp}
        del gR, gI

    # ---- CPU oracle baseline (rank 0, single GPU only)
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, dt, srs, kept = oracle_sample_rate(objs, wo, args.cpu_sample, keep=True)
        cpu = {"value": rate, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
               "sample": f"{len(srs)} objects spread over the dictionary (r = {srs}, mean {np.mean(srs):.1f}) x "
                         f"{args.n_w} frequencies, {dt:.1f} s"}
        accuracy = accuracy_vs_oracle(wo, kept, *acc_out)
        accuracy["sample"] = "the CPU baseline's objects, every frequency, outputs of the last timed step"
        del kept

    sm_mhz_max = (clk or {}).get("sm_max_mhz", 2070.0)
    peak_tflops = SM_COUNT_NOMINAL * DFMA_PER_CLK_PER_SM * 2 * sm_mhz_max * 1e6 / 1e12
    # the DFMA rate measured on this device in this run (independent FMA chains on every SM)
    fp64_measured, _ = m.mrom_fp64_peak(h)
    st = np.array(stages, dtype=np.float64).mean(axis=0)  # mean ms per stage over the timed steps
    achieved = flops_pen / (st[2] * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": SWEEP_DRAM_BYTES_PER_LAUNCH,
                "kernel": "pencil_sweep_kernel", "flops_per_launch": flops_pen,
                "peak_note": "derived FP64 pipe peak: 152 SM x 2 DFMA/clk x 2 flop x max SM clock (no FP64 entry "
                             "in the measured peaks); the DFMA-chain probe mrom_fp64_peak read "
                             f"{fp64_measured:.3f} TFLOP/s in this run"
                             + (", below this kernel's own rate, so the derived figure is the denominator"
                                if fp64_measured < achieved else ""),
                "fp64_probe_in_run": fp64_measured}
    if SWEEP_DRAM_BYTES_PER_LAUNCH is None:
        roofline["traffic_note"] = SWEEP_DRAM_NOTE
    stage_info = {"prep_ms": st[0], "route_ms": st[1], "pencil_sweep_ms": st[2], "lu_sweep_ms": st[3],
                  "prep_flops": flops_prep, "prep_tflops": flops_prep / (st[0] * 1e-3) / 1e12 if st[0] > 0 else None,
                  "objects_pencil": n_pen, "objects_lu": n_lu}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": args.scaling,
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(args),
            "roofline": roofline, "cpu_baseline": cpu, "accuracy_vs_oracle": accuracy, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "wall_s_timed": wall, "per_launch_ms": per_launch_ms, "sweep_config": sweep_cfg,
            "pencil_groups_per_task": pencil_groups,
            "stages": stage_info, "lu_route": lu_route, "mixed_precision": mixed, "projection": proj,
            "gradients": grads, "invariants": inv, "c1_latency": c1, "podp_mu": pmu,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    for x in roms:
        x.close()
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
