"""GPU parity of the PODP in mu_r (mrom_project_mu, mrom_sweep_vjp at per-object s_mu) with
oracle/podp_mu.py.

Both sides keep every snapshot direction (the smallest singular value ratios are 1e-5 for the
12 dynamic and 2e-2 for the 6 static columns, far above the truncation), so the reduced spaces
are the same and the signature, the static quantities and the gradients must agree to
rounding at any (omega, s_mu), not only at the sampled ones; at the sampled ones both also
reproduce the full-order model.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

S_SAMPLES = (1.0, 4.0)
W_SAMPLES = (1e2, 1e4)


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
def case(mrom):
    import torch
    from oracle import podp_mu
    from workloads import fit_problem, full_order_snapshots
    from workloads.fit import Material
    mat = (Material((0.25,) * 3, (0.75,) * 3, 5.96e7, 4.0),)
    probs = {s: fit_problem(8, mat, mu_scale=s, mu_split=True) for s in S_SAMPLES}
    D = [full_order_snapshots(probs[s], W_SAMPLES) for s in S_SAMPLES]
    O = [probs[s].o_tilde for s in S_SAMPLES]
    U, V = podp_mu.bases(D, O, tol_sigma=1e-7, tol_static=1e-7)
    model = podp_mu.project(probs[1.0], U, V)
    h = mrom.Handle(0)
    p1 = probs[1.0]
    fom = mrom.FullOrder.from_fit(p1)
    mu = mrom.PermeabilityData.from_fit(p1, np.concatenate(O, axis=0), tol_static=1e-7)
    cols = np.concatenate([np.transpose(Dl, (2, 0, 1)).reshape(-1, p1.N) for Dl in D], axis=0)
    rom, r, m = mrom.mrom_project_mu(h, fom, mu, torch.as_tensor(np.ascontiguousarray(cols), device="cuda"),
                                     tol_sigma=1e-7)
    return dict(h=h, rom=rom, r=r, m=m, model=model, probs=probs, U=U, V=V)


def test_ranks_match_oracle(case):
    assert case["r"] == case["U"].shape[1] == 12
    assert case["m"] == case["V"].shape[1] == 6


def test_static_state_matches_oracle(mrom, case):
    from oracle import podp_mu
    for s in (0.6, 1.0, 2.2, 4.0, 11.0):
        g = mrom.mrom_rom_mu_state(case["rom"], s)
        o = podp_mu.static_state(case["model"], s)
        for k in ("c00", "N0", "dc00", "dN0"):
            sc = np.abs(o[k]).max()
            assert np.abs(g[k] - o[k]).max() <= 1e-10 * sc, (s, k)
        # B is basis-dependent; its Gram B^H C_r^-1 B is not
        C = case["model"].C
        sc = np.abs(o["B"].conj().T @ np.linalg.solve(C, o["B"])).max()
        Cg = mrom.mrom_rom_get(case["rom"], with_gram=False)["C"]
        dg = g["B"].conj().T @ np.linalg.solve(Cg, g["B"]) - o["B"].conj().T @ np.linalg.solve(C, o["B"])
        assert np.abs(dg).max() <= 1e-8 * sc, s


def _sweep(mrom, case, wo, s_mu, s_sigma, gR, gI, lu):
    import torch
    h = case["h"]
    h.set_solver(lu=lu)
    n = len(s_mu)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    R = torch.empty((n, wo.size, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    g_w = torch.empty((n, wo.size), dtype=torch.float64, device="cuda")
    g_s = torch.empty(n, dtype=torch.float64, device="cuda")
    g_m = torch.empty(n, dtype=torch.float64, device="cuda")
    mrom.mrom_sweep_vjp(h, [case["rom"]] * n, t(wo), wo.size, t(gR), t(gI), g_w, g_ssigma=g_s, g_smu=g_m,
                        s_sigma=t(s_sigma), s_mu=t(s_mu), R=R, I=I)
    h.synchronize()
    h.set_solver(lu=False)
    return R.cpu().numpy(), I.cpu().numpy(), g_w.cpu().numpy(), g_s.cpu().numpy(), g_m.cpu().numpy()


@pytest.mark.parametrize("lu", [False, True], ids=["auto", "lu"])
def test_signature_and_gradients_match_oracle(mrom, case, lu):
    from oracle import podp_mu
    from workloads import log_omegas
    model = case["model"]
    wo = log_omegas(1e1, 1e5, 23)
    s_mu = np.array([0.7, 1.0, 2.3, 4.0, 9.0])
    s_sigma = np.array([1.0, 1.3, 0.8, 1.0, 2.0])
    rng = np.random.default_rng(5)
    gR = rng.standard_normal((s_mu.size, wo.size, 3, 3))
    gI = rng.standard_normal((s_mu.size, wo.size, 3, 3))
    R, I, g_w, g_s, g_m = _sweep(mrom, case, wo, s_mu, s_sigma, gR, gI, lu)
    a3 = model.alpha ** 3
    for k, (sm, ss) in enumerate(zip(s_mu, s_sigma)):
        Rr, Ir = podp_mu.signature(model, wo, s_mu=sm, s_sigma=ss)
        # per frequency: R against max |R~|, I against its term scale w' a^3/4 max |c00(s)|
        # (I is a difference of terms of that size at high omega)
        sR = np.abs(Rr).reshape(wo.size, -1).max(1)
        sI = wo * ss * a3 / 4 * np.abs(podp_mu.static_state(model, sm)["c00"]).max()
        eR = (np.abs(R[k] - Rr).reshape(wo.size, -1).max(1) / sR).max()
        eI = (np.abs(I[k] - Ir).reshape(wo.size, -1).max(1) / sI).max()
        assert eR <= 1e-10 and eI <= 1e-10, (k, eR, eI)
        dR, dI = podp_mu.tangent_s_mu(model, wo, s_mu=sm, s_sigma=ss)
        # dL/ds_mu is a sum over the frequencies, compared relative to the sum of its terms'
        # magnitudes.  Floor 1e-8 (measured 8.7e-9): the two sides' reduced models come from their
        # own truncated SVDs and projections of the same snapshots, and the derivative through the
        # reduced static state (dy/ds, dB/ds, dc00/ds, dN0/ds) amplifies their 1e-11 difference.
        per_w = np.sum(gR[k] * dR, axis=(1, 2)) + np.sum(gI[k] * dI, axis=(1, 2))
        ref, scale = float(per_w.sum()), float(np.abs(per_w).sum())
        assert abs(g_m[k] - ref) <= 1e-8 * scale, (k, g_m[k], ref, scale)


def test_sampled_parameters_reproduce_the_full_order_model(mrom, case):
    from oracle import fom
    wo = np.asarray(W_SAMPLES)
    s_mu = np.asarray(S_SAMPLES)
    z = np.zeros((s_mu.size, wo.size, 3, 3))
    R, I, *_ = _sweep(mrom, case, wo, s_mu, np.ones(s_mu.size), z, z, False)
    for k, s in enumerate(S_SAMPLES):
        p = case["probs"][s]
        Rf, If = fom.fmm_signature(p, wo)
        Rf = Rf + p.N0[None]
        sc = max(np.abs(Rf).max(), np.abs(If).max())
        assert max(np.abs(R[k] - Rf).max(), np.abs(I[k] - If).max()) <= 1e-8 * sc


def test_invalid_scale_is_refused(mrom, case):
    import torch
    with pytest.raises(mrom.MromError):
        mrom.mrom_rom_mu_state(case["rom"], -1.0)
    wo = np.array([1e3])
    z = np.zeros((1, 1, 3, 3))
    with pytest.raises(mrom.MromError):
        _sweep(mrom, case, wo, np.array([0.0]), np.ones(1), z, z, True)
    case["h"].set_solver(lu=False)


def test_two_material_object_matches_oracle(mrom):
    """Shell (mu_r = 1) around a mu_r = 64 core, both scaled by s, snapshots at s = 0.5 and 2
    (smallest singular value ratios 6e-5 dynamic, 0.3 static: both sides keep every direction)."""
    import torch
    from oracle import podp_mu
    from workloads import TWO_MATERIAL_C5, fit_problem, full_order_snapshots, log_omegas
    S = (0.5, 2.0)
    probs = {s: fit_problem(8, TWO_MATERIAL_C5, mu_scale=s, mu_split=True) for s in S}
    p1 = fit_problem(8, TWO_MATERIAL_C5, mu_split=True)
    D = [full_order_snapshots(probs[s], W_SAMPLES) for s in S]
    O = [probs[s].o_tilde for s in S]
    U, V = podp_mu.bases(D, O, tol_sigma=1e-7, tol_static=1e-7)
    model = podp_mu.project(p1, U, V)
    h = mrom.Handle(0)
    fom = mrom.FullOrder.from_fit(p1)
    mu = mrom.PermeabilityData.from_fit(p1, np.concatenate(O, axis=0), tol_static=1e-7)
    cols = np.concatenate([np.transpose(Dl, (2, 0, 1)).reshape(-1, p1.N) for Dl in D], axis=0)
    rom, r, m = mrom.mrom_project_mu(h, fom, mu, torch.as_tensor(np.ascontiguousarray(cols), device="cuda"),
                                     tol_sigma=1e-7)
    assert r == U.shape[1] and m == V.shape[1]
    case = dict(h=h, rom=rom)
    wo = log_omegas(1e1, 1e5, 17)
    s_mu = np.array([0.5, 0.9, 2.0, 3.1])
    s_sigma = np.ones(s_mu.size)
    rng = np.random.default_rng(11)
    gR = rng.standard_normal((s_mu.size, wo.size, 3, 3))
    gI = rng.standard_normal((s_mu.size, wo.size, 3, 3))
    R, I, _, _, g_m = _sweep(mrom, case, wo, s_mu, s_sigma, gR, gI, False)
    a3 = model.alpha ** 3
    for k, sm in enumerate(s_mu):
        Rr, Ir = podp_mu.signature(model, wo, s_mu=sm)
        sR = np.abs(Rr).reshape(wo.size, -1).max(1)
        sI = wo * a3 / 4 * np.abs(podp_mu.static_state(model, sm)["c00"]).max()
        eR = (np.abs(R[k] - Rr).reshape(wo.size, -1).max(1) / sR).max()
        eI = (np.abs(I[k] - Ir).reshape(wo.size, -1).max(1) / sI).max()
        assert eR <= 1e-10 and eI <= 1e-10, (k, eR, eI)
        dR, dI = podp_mu.tangent_s_mu(model, wo, s_mu=sm)
        per_w = np.sum(gR[k] * dR, axis=(1, 2)) + np.sum(gI[k] * dI, axis=(1, 2))
        ref, scale = float(per_w.sum()), float(np.abs(per_w).sum())
        assert abs(g_m[k] - ref) <= 1e-8 * scale, (k, g_m[k], ref, scale)


@pytest.mark.parametrize("lu", [False, True], ids=["auto", "lu"])
def test_sweep_with_certificate_at_scales_matches_oracle(mrom, lu):
    """mrom_sweep at per-object s_mu: R, I and the certificate Delta of Lemma 4.2 at the scale
    (extended Gram of [C x | C V | (K_out + eps M) U | K_in U | C U]) against the oracle; Delta
    per frequency against its term scale (the Gram form cancels terms of that size)."""
    import torch
    from oracle import podp_mu
    from workloads import fit_problem, full_order_snapshots, log_omegas
    from workloads.fit import Material
    mat = (Material((0.25,) * 3, (0.75,) * 3, 5.96e7, 4.0),)
    probs = {s: fit_problem(8, mat, mu_scale=s, mu_split=True) for s in S_SAMPLES}
    p1 = probs[1.0]
    X = p1.eps * p1.M + 10.0 * p1.C
    D = [full_order_snapshots(probs[s], W_SAMPLES) for s in S_SAMPLES]
    O = [probs[s].o_tilde for s in S_SAMPLES]
    U, V = podp_mu.bases(D, O, tol_sigma=1e-7, tol_static=1e-7)
    model = podp_mu.project(p1, U, V)
    podp_mu.attach_extended_gram(model, p1, U, V, X)
    h = mrom.Handle(0)
    h.set_solver(lu=lu)
    fom = mrom.FullOrder.from_fit(p1, X=X)
    mu = mrom.PermeabilityData.from_fit(p1, np.concatenate(O, axis=0), tol_static=1e-7)
    cols = np.concatenate([np.transpose(Dl, (2, 0, 1)).reshape(-1, p1.N) for Dl in D], axis=0)
    rom, r, m = mrom.mrom_project_mu(h, fom, mu, torch.as_tensor(np.ascontiguousarray(cols), device="cuda"),
                                     tol_sigma=1e-7)
    wo = log_omegas(1e1, 1e5, 19)
    s_mu = np.array([0.7, 1.0, 2.3, 4.0, 9.0, 1.8])
    s_sigma = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.6])   # the last instance scales sigma as well
    n = s_mu.size
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    R = torch.empty((n, wo.size, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    Dg = torch.empty_like(R)
    mrom.mrom_sweep(h, [rom] * n, t(wo), wo.size, R, I, Dg, s_mu=t(s_mu), s_sigma=t(s_sigma))
    h.synchronize()
    R, I, Dg = R.cpu().numpy(), I.cpu().numpy(), Dg.cpu().numpy()
    a3 = model.alpha ** 3
    for k, (sm, ss) in enumerate(zip(s_mu, s_sigma)):
        Rr, Ir = podp_mu.signature(model, wo, s_mu=sm, s_sigma=ss)
        Dr = podp_mu.certificate(model, wo, s_mu=sm, s_sigma=ss)
        sR = np.abs(Rr).reshape(wo.size, -1).max(1)
        sI = wo * ss * a3 / 4 * np.abs(podp_mu.static_state(model, sm)["c00"]).max()
        sD = podp_mu.certificate_term_scale(model, wo, s_mu=sm, s_sigma=ss)
        eR = (np.abs(R[k] - Rr).reshape(wo.size, -1).max(1) / sR).max()
        eI = (np.abs(I[k] - Ir).reshape(wo.size, -1).max(1) / sI).max()
        eD = (np.abs(Dg[k] - Dr).reshape(wo.size, -1).max(1) / sD).max()
        assert eR <= 1e-10 and eI <= 1e-10 and eD <= 1e-10, (k, eR, eI, eD)
    # at s = 1 the scaled sweep equals the plain one (the object's stored state is that of s = 1)
    R1, I1, D1 = (torch.empty((1, wo.size, 3, 3), dtype=torch.float64, device="cuda") for _ in range(3))
    mrom.mrom_sweep(h, [rom], t(wo), wo.size, R1, I1, D1)
    h.synchronize()
    sc = np.abs(D1.cpu().numpy()).max()
    assert np.abs(D1.cpu().numpy()[0] - Dg[1]).max() <= 1e-12 * sc
    h.set_solver(lu=False)
    with pytest.raises(mrom.MromError):       # no extended Gram: no certificate at a scale
        plain = mrom.ReducedObject.from_workload(h, __import__("workloads").reduced_object(20230711, 1, 12))
        mrom.mrom_sweep(h, [plain], t(wo), wo.size, R1, I1, D1, s_mu=t([2.0]))


def test_sweep_values_at_scales_without_certificate(mrom, case):
    """mrom_sweep with s_mu (values only) on an object projected without a certificate inner
    product gives the oracle's R and I at each scale, as mrom_sweep_vjp does."""
    import torch
    from oracle import podp_mu
    from workloads import log_omegas
    model = case["model"]
    wo = log_omegas(1e1, 1e5, 13)
    s_mu = np.array([0.6, 2.5, 7.0])
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    h = case["h"]
    R = torch.empty((s_mu.size, wo.size, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    mrom.mrom_sweep(h, [case["rom"]] * s_mu.size, t(wo), wo.size, R, I, s_mu=t(s_mu))
    h.synchronize()
    a3 = model.alpha ** 3
    for k, sm in enumerate(s_mu):
        Rr, Ir = podp_mu.signature(model, wo, s_mu=sm)
        eR = (np.abs(R[k].cpu().numpy() - Rr).reshape(wo.size, -1).max(1) / np.abs(Rr).reshape(wo.size, -1).max(1)).max()
        sI = wo * a3 / 4 * np.abs(podp_mu.static_state(model, sm)["c00"]).max()
        eI = (np.abs(I[k].cpu().numpy() - Ir).reshape(wo.size, -1).max(1) / sI).max()
        assert eR <= 1e-10 and eI <= 1e-10, (k, eR, eI)
