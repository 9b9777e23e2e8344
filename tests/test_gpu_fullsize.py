"""Parity at the full configuration sizes, in the launch configuration bench.py uses.

* 16^3 copper cube, nine snapshots in [1e1, 1e5], 100 outputs: the paper's PODP (one TSVD
  per direction) on the GPU against the oracle, every output.
* 1000 objects x 2000 frequencies (the benchmark dictionary, plan + autotuned launch): sampled
  (object, frequency) pairs recomputed by the oracle one by one; gradients on sampled objects.
* 96^3 grid (N = 2.6M) with 3 x 32 snapshot columns: projection onto the oracle's basis compared
  entry by entry with the oracle's projection, and sampled frequencies of the sweep.
"""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def mrom():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_05590_gb300 import build
    build.build()
    import paper_2307_05590_gb300 as m
    return m


def _scales(model, wo, P):
    from oracle import certificate
    a3 = model.alpha ** 3
    cmax = max(np.abs(model.C[i][j]).max() for i in range(3) for j in range(3))
    bmax = max(np.abs(model.oCU[i][j]).max() for i in range(3) for j in range(3))
    sI, sD = [], []
    for n, w in enumerate(wo):
        pn = sum(np.abs(P[i][n]).sum() for i in range(3))
        sI.append(w * a3 / 4 * (np.abs(model.c00).max() + cmax * pn * pn + 2 * bmax * pn))
        W = certificate.residual_weights(model, w, [P[i][n] for i in range(3)])
        sD.append(a3 / (4 * model.alpha_lb) * max(np.abs(x) @ np.abs(model.gram) @ np.abs(x) for x in W))
    return np.array(sI), np.array(sD)


def test_c1_cube_per_direction_podp(mrom):
    import torch
    from oracle import certificate, rom, tsvd
    from workloads import CUBE_C1, fit_problem, full_order_snapshots, log_omegas
    from gpu_common import rel_errors
    p = fit_problem(16, CUBE_C1)
    ws = log_omegas(1e1, 1e5, 9)
    D = full_order_snapshots(p, ws)                            # (3, N, 9)
    X = p.eps * p.M + 10.0 * p.C
    Us = [tsvd.truncated_svd(D[i], 1e-6)[0] for i in range(3)]
    model = rom.project(p, Us)
    certificate.attach_gram(model, p, Us, sp.diags(X).tocsc())
    wo = log_omegas(1e1, 1e5, 100)
    P = rom.reduced_solve(model, wo)
    Rr, Ir = rom.mm_tensors(model, wo, P)
    Dr = certificate.certificate(model, wo, P)
    sI, sD = _scales(model, wo, P)
    h = mrom.Handle(0)
    fom = mrom.FullOrder.from_fit(p, X=X)
    cols = torch.as_tensor(np.ascontiguousarray(np.concatenate([D[i].T for i in range(3)])), device="cuda")
    obj, sig, rd = mrom.mrom_project_dirs(h, fom, cols, tol_sigma=1e-6)
    assert rd == tuple(U.shape[1] for U in Us)
    om = torch.as_tensor(wo, device="cuda")
    R = torch.empty((1, 100, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    Dg = torch.empty_like(R)
    mrom.mrom_sweep(h, [obj], om, 100, R, I, Dg)
    h.synchronize()
    errs = rel_errors(R[0].cpu().numpy(), I[0].cpu().numpy(), Dg[0].cpu().numpy(), Rr, Ir, Dr, sI, sD)
    assert max(errs) <= TOL, errs


def test_dictionary_1000x2000_sampled(mrom):
    import torch
    from oracle import certificate, grads, rom
    from workloads import log_omegas, reduced_dictionary
    from gpu_common import oracle_sweep, rel_errors
    objs = reduced_dictionary(1000, seed=20230711)
    wo = log_omegas(1e1, 1e8, 2000)
    h = mrom.Handle(0)
    roms = [mrom.ReducedObject.from_workload(h, o) for o in objs]
    mrom.mrom_tune(h, roms, 2000)
    plan = mrom.Plan(h, roms, 2000)
    om = torch.as_tensor(wo, device="cuda")
    R = torch.empty((1000, 2000, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    D = torch.empty_like(R)
    plan.sweep(om, R, I, D)
    h.synchronize()
    rng = np.random.default_rng(7)
    oi = rng.integers(0, 1000, 40)
    wi = rng.integers(0, 2000, 40)
    for o, k in zip(oi, wi):
        ref = oracle_sweep(objs[o], wo[k:k + 1])
        got = [x[o, k:k + 1].cpu().numpy() for x in (R, I, D)]
        assert max(rel_errors(*got, *ref)) <= TOL, (o, k, objs[o].r)
    # gradients on the same dictionary (sampled objects, every frequency)
    sel = [int(x) for x in rng.choice(1000, 6, replace=False)]
    rs = [roms[k] for k in sel]
    gR = torch.as_tensor(rng.standard_normal((6, 2000, 3, 3)), device="cuda")
    gI = torch.as_tensor(rng.standard_normal((6, 2000, 3, 3)), device="cuda")
    g_w = torch.empty((6, 2000), dtype=torch.float64, device="cuda")
    g_s = torch.empty(6, dtype=torch.float64, device="cuda")
    g_m = torch.empty(6, dtype=torch.float64, device="cuda")
    mrom.mrom_sweep_vjp(h, rs, om, 2000, gR, gI, g_w, g_ssigma=g_s, g_smu=g_m)
    h.synchronize()
    for j, k in enumerate(sel):
        dR, dI = grads.tangents(objs[k], wo)
        contrib = np.einsum("twij,wij->tw", dR, gR[j].cpu().numpy()) + \
            np.einsum("twij,wij->tw", dI, gI[j].cpu().numpy())
        # g_omega per (object, omega) against max |g_omega| of the object; the scale derivatives
        # (sums over the 2000 frequencies) against the sum of their terms' magnitudes
        assert np.abs(g_w[j].cpu().numpy() - contrib[0]).max() <= TOL * np.abs(contrib[0]).max()
        assert abs(g_s[j].item() - contrib[1].sum()) <= TOL * np.abs(contrib[1]).sum()
        assert abs(g_m[j].item() - contrib[2].sum()) <= TOL * np.abs(contrib[2]).sum()


def test_c2_grid_projection_full_size(mrom):
    """N = 2,599,200: the GPU projects onto the oracle's TSVD basis; K_r, C_r, eps M_r, b, c00 and
    the certificate Gram are compared entry by entry with the oracle's projection, and 20
    sampled output frequencies of the sweep with the oracle's reduced solve."""
    import torch
    from oracle import certificate, rom, tsvd
    from workloads import CUBE_C2, fit_problem, log_omegas, synthetic_snapshot_matrix
    from gpu_common import oracle_model_sweep, rel_errors
    p = fit_problem(96, CUBE_C2, static=False)
    D = synthetic_snapshot_matrix(p.N, 32, 20230711)
    cols = np.ascontiguousarray(D.transpose(0, 2, 1).reshape(96, p.N))
    del D
    U, s, _, _ = tsvd.truncated_svd(cols.T, 1e-6)
    X = p.eps * p.M + 10.0 * p.C
    model = rom.project(p, U)
    certificate.attach_gram(model, p, U, sp.diags(X).tocsc())
    h = mrom.Handle(0)
    fom = mrom.FullOrder.from_fit(p, X=X)
    obj, _, r = mrom.mrom_project(h, fom, basis=torch.as_tensor(np.ascontiguousarray(U), device="cuda"))
    got = mrom.mrom_rom_get(obj)
    B = np.stack([model.b(i) for i in range(3)], 1)
    for key, ref in (("K", model.K[0][0]), ("C", model.C[0][0]), ("Me", model.Me[0]), ("B", B),
                     ("c00", model.c00), ("G", model.gram)):
        assert np.abs(got[key] - ref).max() <= 1e-12 * np.abs(ref).max(), key
    wo = log_omegas(1e1, 1e8, 10000)[::500]
    om = torch.as_tensor(wo, device="cuda")
    R = torch.empty((1, wo.size, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    Dg = torch.empty_like(R)
    mrom.mrom_sweep(h, [obj], om, wo.size, R, I, Dg)
    h.synchronize()
    errs = rel_errors(R[0].cpu().numpy(), I[0].cpu().numpy(), Dg[0].cpu().numpy(), *oracle_model_sweep(model, wo))
    assert max(errs) <= TOL, errs
