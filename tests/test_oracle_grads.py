"""Pins of the oracle's derivatives (no counterpart in the paper)."""
import numpy as np
import pytest

from oracle import grads, rom
from workloads import log_omegas, reduced_object


@pytest.fixture(scope="module")
def obj():
    return reduced_object(20230711, 3, 14)


def test_forward_matches_rom(obj):
    wo = log_omegas(1e1, 1e8, 9)
    R1, I1 = grads.forward(obj, wo)
    R2, I2, _ = rom.rom_signature(rom.from_reduced_object(obj), wo)
    assert np.abs(R1 - R2).max() <= 1e-12 * np.abs(R2).max()
    assert np.abs(I1 - I2).max() <= 1e-12 * np.abs(I2).max()


@pytest.mark.parametrize("which", [0, 1, 2])
def test_tangents_match_central_differences(obj, which):
    wo = log_omegas(1e1, 1e8, 7) * 1.1
    s_sigma, s_mu = 1.3, 4.0
    dR, dI = grads.tangents(obj, wo, s_sigma, s_mu)
    fR, fI = grads.central_difference(obj, wo, which, 1e-6, s_sigma, s_mu)
    R, I = grads.forward(obj, wo, s_sigma, s_mu)
    theta = [wo, np.full(wo.size, s_sigma), np.full(wo.size, s_mu)][which]
    K = obj.K_out + obj.K_in / s_mu
    for n in range(wo.size):
        # truncation O(h^2) plus the rounding noise of a difference quotient,
        # ~eps * (term scale) / (h theta); I's terms cancel at high omega, so its
        # scale is that of the summands, not of I itself
        A = K - 1j * wo[n] * s_sigma * obj.C
        P = np.linalg.solve(A, 1j * wo[n] * s_sigma * obj.B)
        pn = np.linalg.norm(P)
        termR = np.linalg.norm(K, 2) * pn ** 2 / 4
        termI = wo[n] * s_sigma / 4 * (np.abs(obj.c00).max() + np.linalg.norm(obj.C, 2) * pn ** 2
                                       + 2 * np.linalg.norm(obj.B) * pn)
        noiseR = 1e-9 * termR / theta[n]
        noiseI = 1e-9 * termI / theta[n]
        assert np.abs(dR[which, n] - fR[n]).max() <= 1e-6 * np.abs(dR[which, n]).max() + noiseR
        assert np.abs(dI[which, n] - fI[n]).max() <= 1e-6 * np.abs(dI[which, n]).max() + noiseI


def test_sigma_derivative_equals_omega_derivative(obj):
    """M(w; s sigma) = M(s w; sigma) (nu is linear in w sigma), so d/ds_sigma = w d/dw at s = 1."""
    wo = log_omegas(1e1, 1e8, 11)
    dR, dI = grads.tangents(obj, wo)
    assert np.abs(dR[1] - wo[:, None, None] * dR[0]).max() <= 1e-10 * np.abs(dR[1]).max()
    assert np.abs(dI[1] - wo[:, None, None] * dI[0]).max() <= 1e-10 * np.abs(dI[1]).max()


def test_vjp_contracts_tangents(obj):
    wo = log_omegas(1e1, 1e8, 5)
    rng = np.random.default_rng(1)
    gR = rng.standard_normal((5, 3, 3))
    gI = rng.standard_normal((5, 3, 3))
    gw, gs, gm = grads.vjp(obj, wo, gR, gI, 1.2, 2.0)
    dR, dI = grads.tangents(obj, wo, 1.2, 2.0)
    for n in range(5):
        ref = np.sum(dR[0, n] * gR[n]) + np.sum(dI[0, n] * gI[n])
        assert gw[n] == pytest.approx(ref, rel=1e-12)
    assert gs == pytest.approx(np.sum(dR[1] * gR) + np.sum(dI[1] * gI), rel=1e-12)
    assert gm == pytest.approx(np.sum(dR[2] * gR) + np.sum(dI[2] * gI), rel=1e-12)
