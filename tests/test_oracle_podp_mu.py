"""Pins of the PODP in mu_r (oracle/podp_mu.py) against the full-order model.

At a sampled (omega_k, s_l) whose snapshots are in the bases, Galerkin projection reproduces
the full-order solutions exactly (the reduced spaces contain them), so the reduced R~ and I
must equal the full-order ones of Eqs. (11)-(12) on the problem assembled at mu_r scaled by
s_l; the static quantities likewise.  A dropped or mis-signed term of K(s), b(s), c00(s) or
N0(s) fails there.  Derivatives are pinned by central differences, and the conductivity
reading by the exact identity M(omega; t sigma) = M(t omega; sigma).
"""
import numpy as np
import pytest

from oracle import fom, podp_mu
from workloads import fit_problem, full_order_snapshots
from workloads.fit import Material

MAT = (Material((0.25,) * 3, (0.75,) * 3, 5.96e7, 4.0),)
S_SAMPLES = (1.0, 3.0)
W_SAMPLES = (1e2, 1e4)


@pytest.fixture(scope="module")
def setup():
    probs = {s: fit_problem(6, MAT, mu_scale=s, mu_split=True) for s in S_SAMPLES}
    D = [full_order_snapshots(probs[s], W_SAMPLES) for s in S_SAMPLES]
    O = [probs[s].o_tilde for s in S_SAMPLES]
    U, V = podp_mu.bases(D, O, tol_sigma=1e-13, tol_static=1e-13)
    model = podp_mu.project(probs[1.0], U, V)
    return probs, U, V, model


def _fom(p, omegas):
    R, I = fom.fmm_signature(p, omegas)
    return R + p.N0[None], I


def test_bases_span_the_snapshots(setup):
    probs, U, V, model = setup
    assert U.shape[1] == 3 * len(S_SAMPLES) * len(W_SAMPLES) and V.shape[1] == 3 * len(S_SAMPLES)
    assert np.allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-12)


def test_static_quantities_exact_at_sampled_mu(setup):
    probs, U, V, model = setup
    for s, p in probs.items():
        st = podp_mu.static_state(model, s)
        o_t = np.real(V @ st["y"]).T                       # 3 x N
        assert np.abs(o_t - p.o_tilde).max() <= 1e-9 * np.abs(p.o_tilde).max()
        o = p.x + p.o_tilde
        assert np.allclose(st["c00"], o @ (p.C[:, None] * o.T), rtol=1e-10, atol=1e-14 * np.abs(o).max() ** 2)
        assert np.allclose(st["N0"], p.N0, rtol=1e-9, atol=1e-12 * np.abs(p.N0).max())
        assert np.allclose(st["B"], U.conj().T @ (p.C[:, None] * o.T), rtol=1e-9,
                           atol=1e-12 * np.abs(st["B"]).max())


def test_signature_exact_at_sampled_parameters(setup):
    probs, U, V, model = setup
    for s, p in probs.items():
        R, I = podp_mu.signature(model, W_SAMPLES, s_mu=s)
        Rf, If = _fom(p, W_SAMPLES)
        scale = max(np.abs(Rf).max(), np.abs(If).max())
        assert np.abs(R - Rf).max() <= 1e-9 * scale, s
        assert np.abs(I - If).max() <= 1e-9 * scale, s


def test_signature_between_samples_is_an_approximation(setup):
    """Off the sampled parameters the model is not exact but stays close (sanity, not a pin)."""
    probs, U, V, model = setup
    p = fit_problem(6, MAT, mu_scale=1.7, mu_split=True)
    w = np.array([3e2, 3e3])
    R, I = podp_mu.signature(model, w, s_mu=1.7)
    Rf, If = _fom(p, w)
    scale = max(np.abs(Rf).max(), np.abs(If).max())
    err = max(np.abs(R - Rf).max(), np.abs(I - If).max()) / scale
    assert 1e-12 < err < 0.2


def test_mu_one_object_reduces_to_the_scalar_reading():
    """With mu_r = 1 on B at s = 1 the static field vanishes (o~ = 0, N0 = 0)."""
    mat = (Material((0.25,) * 3, (0.75,) * 3, 5.96e7, 1.0),)
    probs = {s: fit_problem(6, mat, mu_scale=s, mu_split=True) for s in (1.0, 2.0)}
    assert np.abs(probs[1.0].o_tilde).max() == 0.0 and np.abs(probs[2.0].o_tilde).max() > 0.0
    D = [full_order_snapshots(probs[s], W_SAMPLES) for s in probs]
    U, V = podp_mu.bases(D, [probs[s].o_tilde for s in probs], 1e-13, 1e-13)
    model = podp_mu.project(probs[1.0], U, V)
    st = podp_mu.static_state(model, 1.0)
    assert np.abs(st["N0"]).max() <= 1e-13 and np.abs(np.real(V @ st["y"])).max() <= 1e-13
    for s, p in probs.items():
        R, I = podp_mu.signature(model, W_SAMPLES, s_mu=s)
        Rf, If = _fom(p, W_SAMPLES)
        scale = max(np.abs(Rf).max(), np.abs(If).max())
        assert max(np.abs(R - Rf).max(), np.abs(I - If).max()) <= 1e-9 * scale


def test_two_material_object_exact_at_sampled_parameters():
    """Shell (mu_r = 1) around a mu_r = 64 core, both scaled by s: the faces between the two
    materials and between the shell and the exterior split K_in by their cells' shares."""
    from workloads import TWO_MATERIAL_C5
    probs = {s: fit_problem(8, TWO_MATERIAL_C5, mu_scale=s, mu_split=True) for s in (0.5, 2.0)}
    D = [full_order_snapshots(probs[s], W_SAMPLES) for s in probs]
    U, V = podp_mu.bases(D, [probs[s].o_tilde for s in probs], 1e-13, 1e-13)
    base = fit_problem(8, TWO_MATERIAL_C5, mu_split=True)
    model = podp_mu.project(base, U, V)
    for s, p in probs.items():
        R, I = podp_mu.signature(model, W_SAMPLES, s_mu=s)
        Rf, If = _fom(p, W_SAMPLES)
        scale = max(np.abs(Rf).max(), np.abs(If).max())
        assert max(np.abs(R - Rf).max(), np.abs(I - If).max()) <= 1e-9 * scale, s


def test_static_derivatives_central_differences(setup):
    _, _, _, model = setup
    s, h = 1.9, 1e-5
    st = podp_mu.static_state(model, s)
    sp, sm = podp_mu.static_state(model, s + h), podp_mu.static_state(model, s - h)
    for k in ("B", "c00", "N0"):
        fd = (sp[k] - sm[k]) / (2 * h)
        assert np.abs(st["d" + k] - fd).max() <= 1e-6 * np.abs(fd).max(), k


def test_signature_tangent_central_differences(setup):
    _, _, _, model = setup
    w = np.array([2e2, 5e3, 4e4])
    # the quotient's rounding noise grows like kappa(A) eps |I| / h (eps M = 1e-6 makes A
    # ill-conditioned) and its truncation error like h^2: h = 1e-3 balances them near 2e-6
    s, h = 2.3, 1e-3
    dR, dI = podp_mu.tangent_s_mu(model, w, s_mu=s, s_sigma=1.3)
    Rp, Ip = podp_mu.signature(model, w, s_mu=s + h, s_sigma=1.3)
    Rm, Im = podp_mu.signature(model, w, s_mu=s - h, s_sigma=1.3)
    assert np.abs(dR - (Rp - Rm) / (2 * h)).max() <= 1e-5 * np.abs(dR).max()
    assert np.abs(dI - (Ip - Im) / (2 * h)).max() <= 1e-5 * np.abs(dI).max()


def test_conductivity_scale_is_a_frequency_scale():
    """nu = alpha^2 mu_0 omega sigma: the full-order tensors at sigma t equal those at omega t,
    and the reduced model with s_sigma = t matches the full-order model at sigma t."""
    t = 2.5
    p = fit_problem(6, MAT, mu_split=True)
    pt = fit_problem(6, MAT, sigma_scale=t, mu_split=True)
    w = np.array([4e1, 4e3])
    Rt, It = _fom(pt, w)
    R1, I1 = _fom(p, w * t)
    scale = max(np.abs(R1).max(), np.abs(I1).max())
    assert max(np.abs(Rt - R1).max(), np.abs(It - I1).max()) <= 1e-10 * scale
    D = [full_order_snapshots(p, w * t)]
    U, V = podp_mu.bases(D, [p.o_tilde], 1e-13, 1e-13)
    model = podp_mu.project(p, U, V)
    R, I = podp_mu.signature(model, w, s_mu=1.0, s_sigma=t)
    assert max(np.abs(R - Rt).max(), np.abs(I - It).max()) <= 1e-9 * scale


def test_certificate_gram_form_matches_the_full_order_residual(setup):
    """w_i^H G_ext w_i equals the X^-1 norm of the explicit full-order residual at any (omega, s),
    and Delta vanishes (to the Gram form's rounding floor) at the sampled parameters."""
    probs, U, V, model = setup
    p1 = probs[1.0]
    X = p1.eps * p1.M + 10.0 * p1.C
    podp_mu.attach_extended_gram(model, p1, U, V, X)
    for w, s in ((3e2, 1.7), (4e3, 0.6), (2e3, 2.5)):
        direct = podp_mu.residual_norms_direct(model, p1, U, V, X, w, s)
        D = podp_mu.certificate(model, [w], s_mu=s)[0]
        a = model.alpha ** 3 / (4.0 * model.alpha_lb)
        assert np.allclose(np.diag(D), a * direct, rtol=1e-7, atol=1e-10 * a * direct.max()), (w, s)
    # the Gram form's rounding floor grows like omega^2: compare at the same frequency
    for s in S_SAMPLES:
        D0 = podp_mu.certificate(model, W_SAMPLES, s_mu=s)
        Dfar = podp_mu.certificate(model, W_SAMPLES, s_mu=1.6 * s)
        for k in range(len(W_SAMPLES)):
            assert np.abs(D0[k]).max() <= 1e-5 * np.abs(Dfar[k]).max(), (s, k)


def test_certificate_off_diagonal_matches_full_order_residual_differences(setup):
    """Delta_ij for i != j at a scale s (Lemma 4.2) equals alpha^3/(8 alpha_LB)(||r_i||^2 + ||r_j||^2
    + ||r_i - r_j||^2) with the three norms from explicit full-order residual vectors; a sign slip
    in the extended Gram's cross term would move Delta_ij by 4 alpha^3/(8 alpha_LB) Re(w_i^H G w_j)."""
    probs, U, V, model = setup
    p1 = probs[1.0]
    X = p1.eps * p1.M + 10.0 * p1.C
    podp_mu.attach_extended_gram(model, p1, U, V, X)
    a = model.alpha ** 3 / (8.0 * model.alpha_lb)
    for w, s in ((3e2, 1.7), (4e3, 0.6), (2e3, 2.5)):
        nrm = podp_mu.residual_norms_direct(model, p1, U, V, X, w, s)
        dif = podp_mu.residual_differences_direct(model, p1, U, V, X, w, s)
        D = podp_mu.certificate(model, [w], s_mu=s)[0]
        expect = a * (nrm[:, None] + nrm[None, :] + dif)
        assert np.allclose(D, expect, rtol=1e-7, atol=1e-10 * expect.max()), (w, s)
        # the cross term is a sizeable part of every off-diagonal entry
        cross = 0.5 * (nrm[:, None] + nrm[None, :] - dif)
        off = ~np.eye(3, dtype=bool)
        assert (4.0 * a * np.abs(cross[off]) > 1e-3 * expect[off]).all(), (w, s)
