"""Pins of the reduced-order oracle: TSVD (Eqs. (13)-(15)), projection and the
Matrix Method (Eqs. (17)-(19)), the pencil second path."""
import numpy as np
import pytest

from oracle import fom, pencil, pipeline, rom, tsvd
from workloads import CUBE_C1, fit_problem, full_order_snapshots, log_omegas, reduced_object


@pytest.fixture(scope="module")
def snap10():
    p = fit_problem(10, CUBE_C1)
    ws = log_omegas(1e1, 1e5, 5)
    return p, ws, full_order_snapshots(p, ws)


def test_truncation_rank_rule():
    s = np.array([1.0, 1e-2, 1e-6, 9.99e-7, 1e-9])
    assert tsvd.truncation_rank(s, 1e-6) == 3
    assert tsvd.truncation_rank(s, 0.0) == 5
    assert tsvd.truncation_rank(s, 1e-6, r_max=2) == 2
    assert tsvd.truncation_rank(np.zeros(3), 1e-6) == 0


def test_truncated_svd_reconstructs():
    rng = np.random.default_rng(0)
    U0 = np.linalg.qr(rng.standard_normal((200, 6)) + 1j * rng.standard_normal((200, 6)))[0]
    V0 = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))[0]
    s0 = np.array([1, 1e-1, 1e-3, 1e-5, 1e-8, 1e-12])
    D = (U0 * s0) @ V0.conj().T
    U, s, Vh, s_all = tsvd.truncated_svd(D, 1e-6)
    assert U.shape == (200, 4)
    assert np.allclose(s_all, s0, rtol=1e-6, atol=1e-15)
    assert np.abs(U.conj().T @ U - np.eye(4)).max() < 1e-13
    assert np.abs((U * s) @ Vh - D).max() <= 1.1e-8


@pytest.mark.parametrize("shared", [False, True])
def test_galerkin_exact_at_snapshots(snap10, shared):
    """With TOL_Sigma = 0 the reduced space contains every snapshot, so the PODP
    solution at a snapshot frequency equals the full-order one (Eqs. (16)-(17))."""
    p, ws, D = snap10
    model, U, _ = pipeline.build_model(p, D, tol_sigma=0.0, shared=shared, with_gram=False)
    Rr, Ir, _ = rom.rom_signature(model, ws)
    Rf, If = fom.fmm_signature(p, ws)
    o = p.o_tilde + p.x
    scaleI = np.max(ws) * p.alpha ** 3 / 4 * np.abs(o @ (p.C[:, None] * o.T)).max()
    assert np.abs(Rr - Rf).max() <= 1e-10 * np.abs(Rf).max()
    assert np.abs(Ir - If).max() <= 1e-10 * scaleI


def test_reduced_energy_identities(snap10):
    """Galerkin: A_r P = i w B gives I = w a^3/4 (c00 - Re P^H C_r P) for a shared basis,
    and Re(p_i^H (K_r + eps M_r) p_i) = -w Im(p_i^H b_i) for every basis choice."""
    p, ws, D = snap10
    wo = log_omegas(1e1, 1e5, 7) * 1.3
    for shared in (True, False):
        model, _, _ = pipeline.build_model(p, D, tol_sigma=1e-8, shared=shared, with_gram=False)
        R, I, P = rom.rom_signature(model, wo)
        for n, w in enumerate(wo):
            for i in range(3):
                pi = P[i][n]
                lhs = np.real(np.vdot(pi, (model.K[i][i] + model.Me[i]) @ pi))
                rhs = -w * np.imag(np.vdot(pi, model.b(i)))
                assert lhs == pytest.approx(rhs, rel=1e-8, abs=1e-14 * abs(lhs))
            if shared:
                Pm = np.stack([P[i][n] for i in range(3)], 1)
                HC = Pm.conj().T @ model.C[0][0] @ Pm
                ref = w * model.alpha ** 3 / 4 * (model.c00 - HC.real)
                assert np.abs(I[n] - ref).max() <= 1e-9 * w * np.abs(model.c00).max()


def test_brute_force_mm_formulas():
    """Eqs. (18), (19) evaluated with explicit loops for a tiny synthetic object."""
    obj = reduced_object(7, 0, 3)
    model = rom.from_reduced_object(obj)
    w = np.array([37.0])
    R, I, P = rom.rom_signature(model, w)
    for i in range(3):
        for j in range(3):
            s = 0j
            t = 0j
            for a in range(3):
                for b in range(3):
                    s += np.conj(P[i][0][a]) * obj.K[a, b] * P[j][0][b]
                    t += np.conj(P[i][0][a]) * obj.C[a, b] * P[j][0][b]
                t += np.conj(obj.B[a, i]) * P[j][0][a] + obj.B[a, j] * np.conj(P[i][0][a])
            assert R[0, i, j] == pytest.approx(-s.real / 4, rel=1e-12)
            assert I[0, i, j] == pytest.approx(37.0 / 4 * (obj.c00[i, j] + t.real), rel=1e-12)
    # and the reduced solve itself
    A = obj.K - 1j * 37.0 * obj.C
    for i in range(3):
        assert np.allclose(A @ P[i][0], 1j * 37.0 * obj.B[:, i], rtol=1e-12, atol=1e-12)


def test_pencil_path_matches_lu():
    """Independent second path (generalized eigenproblem, no LU) agrees with the solve."""
    for idx, r in enumerate((8, 33, 96)):
        model = rom.from_reduced_object(reduced_object(20230711, idx, r))
        wo = log_omegas(1e1, 1e8, 25)
        P1 = rom.reduced_solve(model, wo)
        P2 = pencil.pencil_solve(model, wo)
        for i in range(3):
            assert np.abs(P1[i] - P2[i]).max() <= 1e-10 * np.abs(P1[i]).max()


def test_outputs_invariant_under_basis_rotation(snap10):
    """R, I depend on span(U) only: U -> U Q (Q unitary) leaves them unchanged."""
    p, ws, D = snap10
    model, U, _ = pipeline.build_model(p, D, tol_sigma=1e-8, shared=True, with_gram=False)
    r = U.shape[1]
    rng = np.random.default_rng(3)
    Q = np.linalg.qr(rng.standard_normal((r, r)) + 1j * rng.standard_normal((r, r)))[0]
    model2 = rom.project(p, U @ Q)
    wo = np.array([55.0, 5e3])
    R1, I1, _ = rom.rom_signature(model, wo)
    R2, I2, _ = rom.rom_signature(model2, wo)
    assert np.abs(R1 - R2).max() <= 1e-10 * np.abs(R1).max()
    assert np.abs(I1 - I2).max() <= 1e-10 * np.abs(I1).max()


def test_dictionary_imaginary_part_psd():
    """c00 = Re(B^H C^-1 B) + Z^T Z makes I PSD for every frequency (Eq. (6c): I is a Gram form)."""
    model = rom.from_reduced_object(reduced_object(20230711, 5, 40))
    wo = log_omegas(1e1, 1e8, 50)
    R, I, _ = rom.rom_signature(model, wo)
    for n in range(wo.size):
        assert np.linalg.eigvalsh(I[n]).min() >= -1e-9 * np.abs(I[n]).max()
        assert np.abs(R[n] - R[n].T).max() <= 1e-12 * np.abs(R[n]).max()
