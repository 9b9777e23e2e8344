"""Pins of oracle.invariants (Sect. 1: eigenvalues of R~ and I are rotation invariant)."""
import numpy as np

from oracle import invariants, rom
from workloads import log_omegas, reduced_object


def _rotation(rng):
    Q, R = np.linalg.qr(rng.standard_normal((3, 3)))
    Q = Q * np.sign(np.diag(R))[None, :]
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def test_invariant_under_rotation_of_a_signature():
    """R and I of a reduced object, rotated as Q M Q^T, give the same eigenvalues."""
    obj = reduced_object(5, 1, 20)
    model = rom.from_reduced_object(obj)
    wo = log_omegas(1e1, 1e8, 15)
    P = rom.reduced_solve(model, wo)
    R, I = rom.mm_tensors(model, wo, P)
    rng = np.random.default_rng(2)
    for M in (R, I):
        Q = _rotation(rng)
        Mr = np.einsum("ab,nbc,dc->nad", Q, M, Q)
        e0, e1 = invariants.mpt_invariants(M), invariants.mpt_invariants(Mr)
        assert np.abs(e0 - e1).max() <= 1e-12 * np.abs(e0).max()


def test_closed_forms_and_identities():
    rng = np.random.default_rng(4)
    d = rng.standard_normal((50, 3))
    D = np.zeros((50, 3, 3))
    D[:, [0, 1, 2], [0, 1, 2]] = d
    assert np.array_equal(invariants.mpt_invariants(D), np.sort(d, axis=1))
    A = rng.standard_normal((200, 3, 3))
    S = 0.5 * (A + np.swapaxes(A, 1, 2))
    e = invariants.mpt_invariants(S)
    assert np.allclose(e.sum(axis=1), np.trace(S, axis1=1, axis2=2), rtol=0, atol=1e-13)
    assert np.allclose(e.prod(axis=1), np.linalg.det(S), rtol=1e-12, atol=1e-13)
    assert np.all(np.diff(e, axis=1) >= 0)
    # an object with cubic symmetry has a multiple of the identity (triple eigenvalue)
    assert np.allclose(invariants.mpt_invariants(3.5 * np.eye(3)), 3.5)
    # only the symmetric part counts
    K = np.array([[0.0, 1.0, 0.0], [-1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    assert np.allclose(invariants.mpt_invariants(S[0] + K), e[0])
