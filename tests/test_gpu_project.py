"""GPU parity of mrom_project (snapshot TSVD, Eqs. (13)-(15); projection, Eqs. (17)-(19);
certificate Gram, Lemma 4.2) against the CPU oracle, through the C ABI."""
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


@pytest.fixture(scope="module")
def case():
    """12^3 grid, copper cube [0.25, 0.75]^3, six snapshots in [1e1, 1e5]; diagonal
    certificate inner product X = eps M + omega_min C."""
    from workloads import fit_problem, full_order_snapshots, log_omegas
    from workloads.fit import Material
    p = fit_problem(12, (Material((0.25,) * 3, (0.75,) * 3, 5.96e7, 1.0),))
    ws = log_omegas(1e1, 1e5, 6)
    D = full_order_snapshots(p, ws)
    Dcols = np.ascontiguousarray(np.concatenate(list(D), axis=1).T)  # (18, N): column c contiguous
    X = p.eps * p.M + 10.0 * p.C
    return p, Dcols, X


def _oracle_model(p, Dcols, X, tol):
    from oracle import certificate, rom, tsvd
    U, s, _, s_all = tsvd.truncated_svd(Dcols.T, tol)
    model = rom.project(p, U)
    certificate.attach_gram(model, p, U, sp.diags(X).tocsc())
    return model, U, s_all


def _sweep(mrom, h, roms, wo):
    import torch
    om = torch.as_tensor(wo, device="cuda")
    R = torch.empty((len(roms), wo.size, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    D = torch.empty_like(R)
    mrom.mrom_sweep(h, roms, om, wo.size, R, I, D)
    h.synchronize()
    return R.cpu().numpy(), I.cpu().numpy(), D.cpu().numpy()


def test_projection_onto_given_basis_matches_oracle(mrom, case):
    """Strict parity: the oracle's basis is projected on the GPU (Eqs. (17)-(19), Lemma 4.2)."""
    import torch
    from workloads import log_omegas
    from gpu_common import oracle_model_sweep, rel_errors
    p, Dcols, X = case
    model, U, _ = _oracle_model(p, Dcols, X, 1e-6)
    h = mrom.Handle(0)
    fom = mrom.FullOrder.from_fit(p, X=X)
    Ud = torch.as_tensor(np.ascontiguousarray(U), device="cuda")
    rom, _, r = mrom.mrom_project(h, fom, basis=Ud)
    assert r == U.shape[1]
    got = mrom.mrom_rom_get(rom)
    B = np.stack([model.b(i) for i in range(3)], 1)
    for key, ref in (("K", model.K[0][0]), ("C", model.C[0][0]), ("Me", model.Me[0]), ("B", B),
                     ("c00", model.c00), ("G", model.gram)):
        err = np.abs(got[key] - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, (key, err)
    wo = log_omegas(1e1, 1e5, 64) * 1.03
    Rg, Ig, Dg = _sweep(mrom, h, [rom], wo)
    errs = rel_errors(Rg[0], Ig[0], Dg[0], *oracle_model_sweep(model, wo))
    assert max(errs) <= TOL, errs


def test_gpu_tsvd_matches_oracle(mrom, case):
    """End to end with the GPU's own TSVD.  The cut at TOL_Sigma = 1e-6 has a 232x gap
    (s_12 / s_13), so both sides keep the same subspace; R, I and Delta agree to 1e-10."""
    import torch
    from workloads import log_omegas
    from gpu_common import oracle_model_sweep, rel_errors
    p, Dcols, X = case
    model, U, s_ref = _oracle_model(p, Dcols, X, 1e-6)
    h = mrom.Handle(0)
    fom = mrom.FullOrder.from_fit(p, X=X)
    Dd = torch.as_tensor(Dcols, device="cuda")
    rom, sig, r = mrom.mrom_project(h, fom, Dd, tol_sigma=1e-6)
    assert r == U.shape[1] == 12
    # singular values from the Gram D^H D: absolute accuracy ~ eps s_1^2 / s
    big = s_ref >= 1e-7 * s_ref[0]
    assert np.all(np.abs(sig[big] - s_ref[big]) <= 1e-12 * s_ref[0] ** 2 / s_ref[big] + 1e-12 * s_ref[big])
    wo = log_omegas(1e1, 1e5, 64) * 1.03
    Rg, Ig, Dg = _sweep(mrom, h, [rom], wo)
    errs = rel_errors(Rg[0], Ig[0], Dg[0], *oracle_model_sweep(model, wo))
    assert max(errs) <= TOL, errs


def test_gpu_tsvd_of_a_rank_deficient_snapshot_set(mrom, case):
    """Repeated and linearly combined snapshot columns: the snapshot Gram has a cluster of
    eigenvalues at its rounding level (the eigensolver must still converge, and the retained
    subspace is the oracle's); outputs agree with the oracle's model to 1e-10."""
    import torch
    from workloads import log_omegas
    from gpu_common import oracle_model_sweep, rel_errors
    p, Dcols, X = case
    extra = np.stack([Dcols[0], 2.0 * Dcols[3] - 0.5j * Dcols[7], Dcols[11], Dcols[5] + Dcols[6]])
    Dd_host = np.ascontiguousarray(np.concatenate([Dcols, extra, Dcols[:6]]))  # 28 columns, rank 18
    model, U, _ = _oracle_model(p, Dd_host, X, 1e-6)
    h = mrom.Handle(0)
    fom = mrom.FullOrder.from_fit(p, X=X)
    rom, sig, r = mrom.mrom_project(h, fom, torch.as_tensor(Dd_host, device="cuda"), tol_sigma=1e-6)
    assert r == U.shape[1]
    wo = log_omegas(1e1, 1e5, 48) * 1.03
    Rg, Ig, Dg = _sweep(mrom, h, [rom], wo)
    errs = rel_errors(Rg[0], Ig[0], Dg[0], *oracle_model_sweep(model, wo))
    assert max(errs) <= TOL, errs


def test_project_rejects_bad_input(mrom, case):
    import torch
    p, Dcols, X = case
    h = mrom.Handle(0)
    fom = mrom.FullOrder.from_fit(p, X=X)
    with pytest.raises(mrom.MromError):
        mrom.mrom_project(h, fom, torch.zeros((200, p.N), dtype=torch.complex128, device="cuda"))
    with pytest.raises(mrom.MromError):
        mrom.mrom_project(h, fom, basis=torch.zeros((p.N, 120), dtype=torch.complex128, device="cuda"))


def test_per_direction_bases_match_oracle(mrom, case):
    """The paper's PODP: one TSVD per direction (Sect. 4.1), cross blocks K_ij = U_i^H K U_j in
    Eq. (18), I_ij of Eq. (19) and the certificate with Phi_i = [C o_i | (K+eps M)U_i | C U_i].
    Both with the oracle's bases and with the GPU's own per-direction TSVDs."""
    import torch
    from oracle import certificate, rom, tsvd
    from workloads import log_omegas
    from gpu_common import rel_errors
    p, Dcols, X = case
    n_s = Dcols.shape[0] // 3
    Us = [tsvd.truncated_svd(Dcols[i * n_s:(i + 1) * n_s].T, 1e-6)[0] for i in range(3)]
    model = rom.project(p, Us)
    certificate.attach_gram(model, p, Us, sp.diags(X).tocsc())
    wo = log_omegas(1e1, 1e5, 48) * 1.07
    P = rom.reduced_solve(model, wo)
    Rr, Ir = rom.mm_tensors(model, wo, P)
    Dr = certificate.certificate(model, wo, P)
    a3 = model.alpha ** 3
    # term scales (reading 10): I against w a^3/4 (|c00| + |forms|), Delta against |w|^T |G| |w|
    sI = np.array([w * a3 / 4 * (np.abs(model.c00).max() + sum(np.abs(P[i][n]).sum() ** 2 for i in range(3)) *
                                 max(np.abs(model.C[i][j]).max() for i in range(3) for j in range(3)) +
                                 2 * max(np.abs(model.oCU[i][j]).max() for i in range(3) for j in range(3)) *
                                 sum(np.abs(P[i][n]).sum() for i in range(3))) for n, w in enumerate(wo)])
    absG = np.abs(model.gram)
    sD = np.array([a3 / (4 * model.alpha_lb) * max(np.abs(x) @ absG @ np.abs(x) for x in
                   certificate.residual_weights(model, w, [P[i][n] for i in range(3)])) for n, w in enumerate(wo)])
    h = mrom.Handle(0)
    fom = mrom.FullOrder.from_fit(p, X=X)
    W = torch.as_tensor(np.ascontiguousarray(np.concatenate(Us, axis=1)), device="cuda")
    rd = tuple(U.shape[1] for U in Us)
    obj, _, rd_out = mrom.mrom_project_dirs(h, fom, basis=W, r_dirs=rd)
    assert rd_out == rd
    obj2, sig, rd2 = mrom.mrom_project_dirs(h, fom, torch.as_tensor(Dcols, device="cuda"), tol_sigma=1e-6)
    assert rd2 == rd
    for o in (obj, obj2):
        Rg, Ig, Dg = _sweep(mrom, h, [o], wo)
        errs = rel_errors(Rg[0], Ig[0], Dg[0], Rr, Ir, Dr, sI, sD)
        assert max(errs) <= TOL, errs


def test_mixed_projection_matches_oracle(mrom, case):
    """Single-precision projection products (K U in complex64; K_r, C_r, eps M_r, b on the tensor
    cores with the 3 x TF32 split and FP32 accumulation per CTA, float64 summation of the per-CTA
    partials; TSVD and certificate Gram in float64): the reduced
    tensors stay within the mixed-precision tolerance of 1e-5 of the float64 oracle."""
    import torch
    from workloads import log_omegas
    from gpu_common import oracle_model_sweep, rel_errors
    p, Dcols, X = case
    model, U, _ = _oracle_model(p, Dcols, X, 1e-6)
    h = mrom.Handle(0)
    h.set_projection_precision(True)
    fom = mrom.FullOrder.from_fit(p, X=X)
    Ud = torch.as_tensor(np.ascontiguousarray(U), device="cuda")
    rom, _, r = mrom.mrom_project(h, fom, basis=Ud)
    got = mrom.mrom_rom_get(rom)
    # the certificate Gram is float64 whatever the projection precision
    assert np.abs(got["G"] - model.gram).max() <= 1e-12 * np.abs(model.gram).max()
    # complex64 products: entrywise error bounded by a few ulps of float32 times the
    # magnitude sum |U|^H |A| |U| (row sums of up to a few thousand terms per partial)
    absU = np.abs(U)
    Kabs = abs(p.K)
    B = np.stack([model.b(i) for i in range(3)], 1)
    absO = np.abs(p.o.T)
    for key, ref, mag in (("K", model.K[0][0], absU.T @ (Kabs @ absU)),
                          ("C", model.C[0][0], absU.T @ (p.C[:, None] * absU)),
                          ("Me", model.Me[0], absU.T @ ((p.eps * p.M)[:, None] * absU)),
                          ("B", B, absU.T @ (p.C[:, None] * absO))):
        assert np.all(np.abs(got[key] - ref) <= 1e-5 * mag + 1e-300), key
    wo = log_omegas(1e1, 1e5, 64) * 1.03
    Rg, Ig, Dg = _sweep(mrom, h, [rom], wo)
    eR, eI, eD = rel_errors(Rg[0], Ig[0], Dg[0], *oracle_model_sweep(model, wo))
    assert max(eR, eI) <= 1e-5, (eR, eI)
    assert eD <= 1e-4, eD
