"""Pins of the certificate (Lemma 4.2) and of Algorithm 1."""
import numpy as np
import pytest

from oracle import adapt, certificate, fom, pipeline, rom
from workloads import CUBE_C1, fit_problem, full_order_snapshots, log_omegas, reduced_object


@pytest.fixture(scope="module")
def poor_rom():
    """16^3 copper cube with three snapshots: a deliberately poor ROM whose
    residual is far above the rounding floor of the Gram form."""
    p = fit_problem(16, CUBE_C1)
    ws = log_omegas(1e1, 1e5, 3)
    D = full_order_snapshots(p, ws)
    model, U, _ = pipeline.build_model(p, D, tol_sigma=1e-6, omega_min=10.0)
    return p, U, model


def test_gram_form_equals_residual_norm(poor_rom):
    """w^H G w (Lemma 4.2's fast form) equals rho^H X^-1 rho from the explicit residual."""
    p, U, model = poor_rom
    X = certificate.inner_product_matrix(p, 10.0)
    wo = np.array([13.7, 137.0, 1370.0])
    P = rom.reduced_solve(model, wo)
    for n, w in enumerate(wo):
        direct = certificate.residual_norms_direct(p, U, w, [P[i][n] for i in range(3)], X)
        W = certificate.residual_weights(model, w, [P[i][n] for i in range(3)])
        gram = [np.real(np.vdot(W[i], model.gram @ W[i])) for i in range(3)]
        assert np.allclose(gram, direct, rtol=1e-6)


@pytest.fixture(scope="module")
def skew_rom():
    """12^3 grid with an object of two overlapping boxes that has no mirror plane, so the three
    directions' residuals are not orthogonal and the cross terms of Lemma 4.2 do not vanish;
    two snapshots make a poor ROM whose residual is far above the Gram form's rounding floor."""
    from workloads.fit import Material
    mats = (Material((0.25, 0.25, 0.25), (0.5, 0.75, 0.5), 5.96e7, 1.0),
            Material((0.5, 0.25, 0.4), (0.75, 0.5, 0.75), 5.96e7, 1.0))
    p = fit_problem(12, mats)
    D = full_order_snapshots(p, log_omegas(1e1, 1e5, 2))
    model, U, _ = pipeline.build_model(p, D, tol_sigma=1e-6, omega_min=10.0)
    return p, U, model


def test_off_diagonal_certificate_matches_explicit_residual_differences(skew_rom):
    """Delta_ij for i != j (Lemma 4.2) equals alpha^3/(8 alpha_LB)(||r_i||^2 + ||r_j||^2 + ||r_i - r_j||^2)
    with every norm taken from explicit full-order residual vectors, not from the Gram form.
    Tolerance: 1e-6 relative plus the Gram form's absolute rounding floor 1e-13 |w|^T |G| |w|.
    A flipped sign of the cross term Re(w_i^H G w_j) would move Delta_ij by
    4 alpha^3/(8 alpha_LB) Re(w_i^H G w_j); the test checks that this is far above the tolerance."""
    p, U, model = skew_rom
    X = certificate.inner_product_matrix(p, 10.0)
    wo = np.array([13.7, 210.0, 1370.0])
    P = rom.reduced_solve(model, wo)
    Dl = certificate.certificate(model, wo, P)
    a = model.alpha ** 3 / (8.0 * model.alpha_lb)
    absG = np.abs(model.gram)
    for n, w in enumerate(wo):
        pn = [P[i][n] for i in range(3)]
        nrm = certificate.residual_norms_direct(p, U, w, pn, X)
        dif = certificate.residual_differences_direct(p, U, w, pn, X)
        assert np.abs(np.diag(dif)).max() == 0.0
        expect = a * (nrm[:, None] + nrm[None, :] + dif)
        W = certificate.residual_weights(model, w, pn)
        floor = 1e-13 * 2.0 * a * max(np.abs(x) @ absG @ np.abs(x) for x in W)
        tol = 1e-6 * np.abs(expect) + floor
        assert (np.abs(Dl[n] - expect) <= tol).all(), w
        for i in range(3):
            for j in range(3):
                if i != j:
                    cross = np.real(np.vdot(W[i], model.gram @ W[j]))
                    assert 4.0 * a * abs(cross) > 100.0 * tol[i, j], (w, i, j)


def test_certificate_structure(poor_rom):
    p, U, model = poor_rom
    wo = log_omegas(1e1, 1e5, 9) * 1.2
    P = rom.reduced_solve(model, wo)
    Dl = certificate.certificate(model, wo, P)
    for n, w in enumerate(wo):
        assert np.abs(Dl[n] - Dl[n].T).max() <= 1e-12 * Dl[n].max()
        assert Dl[n].min() > 0.0
        W = certificate.residual_weights(model, w, [P[i][n] for i in range(3)])
        for i in range(3):
            nrm = np.real(np.vdot(W[i], model.gram @ W[i]))
            # ||r_i - r_i|| = 0, so Delta_ii = alpha^3 / (4 alpha_LB) ||r_i||^2
            assert Dl[n, i, i] == pytest.approx(model.alpha ** 3 / (4 * model.alpha_lb) * nrm, rel=1e-9)


def test_certificate_bounds_error_above_lowest_band(poor_rom):
    """Lemma 4.2 used as a bound (empirical under the X / alpha_LB reading): it
    holds for omega >= 10 omega_min on this object; at omega ~ omega_min the
    R error exceeds Delta (recorded as a finding, not tuned away)."""
    p, U, model = poor_rom
    wo = np.array([137.0, 1.37e3, 1.37e4, 9.0e4])
    Rr, Ir, P = rom.rom_signature(model, wo)
    Rf, If = fom.fmm_signature(p, wo)
    Dl = certificate.certificate(model, wo, P)
    err = np.maximum(np.abs(Rr - Rf), np.abs(Ir - If))
    assert np.all(Dl >= err)


def test_certificate_vanishes_at_snapshots():
    """With r = N_s the residual at a snapshot is zero; the Gram form returns it to
    within its rounding floor eps * ||G|| * ||w||^2."""
    p = fit_problem(10, CUBE_C1)
    ws = log_omegas(1e1, 1e5, 4)
    D = full_order_snapshots(p, ws)
    model, U, _ = pipeline.build_model(p, D, tol_sigma=0.0, omega_min=10.0)
    P = rom.reduced_solve(model, ws)
    Dl = certificate.certificate(model, ws, P)
    for n, w in enumerate(ws):
        W = certificate.residual_weights(model, w, [P[i][n] for i in range(3)])
        floor = 1e-13 * np.abs(model.gram).max() * max(np.vdot(x, x).real for x in W)
        assert np.abs(Dl[n]).max() <= floor


def test_interval_maxima_brute_force():
    snaps = np.array([1.0, 10.0, 100.0, 1000.0])
    wo = np.array([1.0, 2.0, 5.0, 10.0, 20.0, 50.0, 99.0, 100.0, 500.0])
    d = np.array([9.0, 1.0, 3.0, 7.0, 2.0, 2.0, 0.5, 8.0, 4.0])
    lam, cand = adapt.interval_maxima(snaps, wo, d)
    # snapshot points (1, 10, 100) are skipped; ties go to the lowest omega
    assert lam.tolist() == [3.0, 2.0, 4.0]
    assert cand.tolist() == [5.0, 20.0, 500.0]


def test_snapshot_selection_fixed_count_and_threshold():
    """The fixed-N_* rule of Algorithm 1 and the variant with a threshold theta (Sect. 4.4):
    empty intervals (Lambda_n = -inf) are never chosen, ties go to the lower interval."""
    lam = np.array([0.4, 1.0, -np.inf, 0.6, 0.5, 0.6])
    cand = np.array([15.0, 25.0, np.nan, 45.0, 55.0, 65.0])
    # fixed count: the N_* largest, returned in ascending frequency
    assert adapt.select_new(lam, cand, 1).tolist() == [25.0]
    assert adapt.select_new(lam, cand, 3).tolist() == [25.0, 45.0, 65.0]
    assert adapt.select_new(lam, cand, 10).tolist() == [15.0, 25.0, 45.0, 55.0, 65.0]
    # threshold: Lambda_n >= theta Lambda (0.5 >= 0.5 included), capped at N_*
    assert adapt.select_new(lam, cand, 10, theta=0.5).tolist() == [25.0, 45.0, 55.0, 65.0]
    assert adapt.select_new(lam, cand, 10, theta=0.55).tolist() == [25.0, 45.0, 65.0]
    assert adapt.select_new(lam, cand, 2, theta=0.5).tolist() == [25.0, 45.0]
    assert adapt.select_new(lam, cand, 10, theta=1.0).tolist() == [25.0]
    assert adapt.select_new(lam, cand, 10, theta=1e-9).tolist() == [15.0, 25.0, 45.0, 55.0, 65.0]


def test_adaptive_loop_threshold_one_is_one_snapshot_per_iteration():
    """theta = 1 keeps only the interval of the largest Lambda_n, so with a unique maximum it
    makes the same choices as N_* = 1, whatever the cap."""
    from workloads.fit import Material
    p = fit_problem(8, (Material((0.25,) * 3, (0.75,) * 3, 5.96e7, 1.0),))
    snap = lambda ws: full_order_snapshots(p, ws)
    wo = log_omegas(1e1, 1e5, 40)
    w0 = log_omegas(1e1, 1e5, 3)
    _, s1, h1, k1 = adapt.adaptive_podp(p, snap, w0, wo, tol_sigma=1e-10, tol_delta=1e-30, n_star=1, max_k=3)
    _, st, ht, kt = adapt.adaptive_podp(p, snap, w0, wo, tol_sigma=1e-10, tol_delta=1e-30, n_star=4, max_k=3,
                                        theta=1.0)
    assert k1 == kt and s1.tolist() == st.tolist()
    assert np.allclose(h1, ht, rtol=1e-12, atol=0.0)


def test_adaptive_loop_grows_and_reduces_lambda():
    """Algorithm 1 with N_* = 2: N grows by two per iteration (Sects. 7.1/7.2 report
    13, 15, 17, 19) and the maximum certificate falls."""
    from workloads.fit import Material
    p = fit_problem(12, (Material((0.25,) * 3, (0.75,) * 3, 5.96e7, 1.0),))
    cache = {}

    def snap(ws):
        out = []
        for w in ws:
            if w not in cache:
                cache[w] = full_order_snapshots(p, [w])[:, :, 0]
            out.append(cache[w])
        return np.stack(out, axis=2)

    wo = log_omegas(1e1, 1e5, 60)
    model, snaps, hist, k = adapt.adaptive_podp(p, snap, log_omegas(1e1, 1e5, 3), wo,
                                                tol_sigma=1e-10, tol_delta=1e-30, n_star=2, max_k=4)
    assert k == 4
    assert snaps.size == 3 + 2 * (k - 1)
    assert len(hist) == k - 1
    assert all(b < 1e-2 * a for a, b in zip(hist, hist[1:]))


def test_dictionary_gram_consistent_with_reduced_residual():
    """For the synthetic object, Phi = U [B|K|C] + Y with U^H Y = 0: the U-part of
    the residual is the Galerkin residual, which vanishes, so w^H G w = ||Y w||^2.
    Checked by rebuilding G from a different Y draw with the same Y^H Y."""
    obj = reduced_object(11, 2, 12)
    model = rom.from_reduced_object(obj)
    wo = np.array([50.0, 5e5])
    P = rom.reduced_solve(model, wo)
    PsiU = np.concatenate([obj.B, obj.K, obj.C], axis=1)
    YhY = obj.G - PsiU.conj().T @ PsiU
    for n, w in enumerate(wo):
        W = certificate.residual_weights(model, w, [P[i][n] for i in range(3)])
        for i in range(3):
            galerkin = PsiU @ W[i]
            assert np.linalg.norm(galerkin) <= 1e-9 * np.linalg.norm(np.abs(PsiU) @ np.abs(W[i]))
            full = np.real(np.vdot(W[i], obj.G @ W[i]))
            orth = np.real(np.vdot(W[i], YhY @ W[i]))
            assert full == pytest.approx(orth, rel=1e-6)
