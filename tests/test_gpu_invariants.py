"""GPU parity of mrom_invariants (rotation invariants of Sect. 1: eigenvalues of R~ and I per
frequency) against oracle.invariants, through the C ABI."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrom():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_05590_gb300 import build
    build.build()
    import paper_2307_05590_gb300 as m
    return m


def _eig(mrom, h, M):
    import torch
    Md = torch.as_tensor(np.ascontiguousarray(M), device="cuda")
    out = torch.empty(Md.shape[:-1], dtype=torch.float64, device="cuda")
    mrom.mrom_invariants(h, Md, out)
    h.synchronize()
    return out.cpu().numpy()


def test_invariants_of_swept_signatures(mrom):
    import torch
    from oracle import invariants
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    objs = [reduced_object(13, k, r) for k, r in enumerate([6, 33, 90])]
    roms = [mrom.ReducedObject.from_workload(h, o) for o in objs]
    wo = log_omegas(1e1, 1e8, 300)
    om = torch.as_tensor(wo, device="cuda")
    R = torch.empty((3, 300, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    mrom.mrom_sweep(h, roms, om, 300, R, I)
    h.synchronize()
    for M in (R.cpu().numpy(), I.cpu().numpy()):
        got = _eig(mrom, h, M)
        ref = invariants.mpt_invariants(M)
        scale = np.abs(ref).max(axis=-1, keepdims=True)
        assert np.all(np.abs(got - ref) <= 1e-13 * scale)


def test_invariants_of_degenerate_and_random_matrices(mrom):
    from oracle import invariants
    h = mrom.Handle(0)
    rng = np.random.default_rng(9)
    A = rng.standard_normal((5000, 3, 3)) * 10.0 ** rng.uniform(-8, 8, (5000, 1, 1))
    Ms = [A,
          np.broadcast_to(np.eye(3) * 2.5, (7, 3, 3)),                      # cubic symmetry
          np.stack([np.diag([1.0, 1.0, -3.0]), np.diag([0.0, 0.0, 0.0]),    # repeated eigenvalues, zero
                    np.diag([5.0, -5.0, 5.0 + 1e-15])])]
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Ms.append(np.einsum("ab,nbc,dc->nad", Q, Ms[2], Q))                  # rotated repeated eigenvalues
    for M in Ms:
        got = _eig(mrom, h, M)
        ref = invariants.mpt_invariants(M)
        scale = np.maximum(np.abs(ref).max(axis=-1, keepdims=True), 1e-300)
        assert np.all(np.abs(got - ref) <= 1e-13 * scale)
    # empty input is a no-op; a negative count is refused
    import torch
    mrom.mrom_invariants(h, torch.empty((0, 3, 3), dtype=torch.float64, device="cuda"),
                         torch.empty((0, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(mrom.MromError):
        mrom._abi.check(mrom.lib().mrom_invariants(h.ptr, None, -1, None), h.ptr)


@pytest.mark.parametrize("lu", [False, True], ids=["pencil", "lu"])
def test_invariants_fused_into_the_sweep(mrom, lu):
    """mrom_plan_sweep_invariants: the eigenvalues of R~ and I computed in the sweep kernels'
    epilogue equal those of the R and I outputs (oracle.invariants on the same values) at 1e-13
    of the matrix scale, on both routes, with an object that carries N0 and Me; with R and I
    omitted the same invariants are written."""
    import torch
    from oracle import invariants
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    h.set_solver(lu=lu)
    objs = [reduced_object(13, k, r) for k, r in enumerate([6, 33, 90])]
    roms = [mrom.ReducedObject.from_workload(h, o) for o in objs]
    o = reduced_object(14, 0, 20)
    rng = np.random.default_rng(4)
    Z = (rng.standard_normal((20, 20)) + 1j * rng.standard_normal((20, 20))) * 1e-3
    N0 = np.array([[0.3, 0.01, 0.0], [0.01, 0.3, 0.02], [0.0, 0.02, 0.25]])
    roms.append(mrom.ReducedObject(h, 20, o.K, o.C, o.B, o.c00, G=o.G, Me=Z @ Z.conj().T, N0=N0))
    n_w = 257
    wo = log_omegas(1e1, 1e8, n_w)
    om = torch.as_tensor(wo, device="cuda")
    plan = mrom.Plan(h, roms, n_w)
    R = torch.empty((len(roms), n_w, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    E = torch.full((len(roms), n_w, 6), float("nan"), dtype=torch.float64, device="cuda")
    plan.sweep(om, R, I, eig=E)
    h.synchronize()
    if not lu:
        assert plan.solver_counts()[0] > 0
    got = E.cpu().numpy()
    for k, M in enumerate((R.cpu().numpy(), I.cpu().numpy())):
        ref = invariants.mpt_invariants(M)
        scale = np.maximum(np.abs(ref).max(axis=-1, keepdims=True), 1e-300)
        assert np.all(np.abs(got[..., 3 * k:3 * k + 3] - ref) <= 1e-13 * scale), k
    E2 = torch.full_like(E, float("nan"))
    plan.sweep(om, None, None, eig=E2)
    h.synchronize()
    assert np.array_equal(E2.cpu().numpy(), got)
    plan.close()
