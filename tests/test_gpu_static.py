"""GPU parity of mrom_static_solve, the regularised static problem behind theta^(0) (Sect. 3,
below Eq. (5)) for a magnetic object, against a sparse direct solve whose gradient part is then
fixed exactly by the nodal problem (the condition G^T M_s o~ = 0 that the solution satisfies)."""
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


@pytest.mark.parametrize("n", [16, 24])
def test_static_solve_matches_direct_solve(mrom, n):
    """mu_r = 32 cube (the 96^3 case's material): o~ entry by entry at 1e-9 of max |o~|, N0 at
    1e-10, and the gradient condition and the residual at the solver's tolerance."""
    import scipy.sparse as sp
    from workloads import CUBE_C2, fit_problem
    from workloads.fit import node_gradient
    p = fit_problem(n, CUBE_C2)                      # direct solve + exact gradient correction
    h = mrom.Handle(0)
    solver = mrom.static_solver_for(h, n)
    q = fit_problem(n, CUBE_C2, static_solver=solver)
    ref, got = p.o_tilde, q.o_tilde
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    assert np.abs(q.N0 - p.N0).max() <= 1e-10 * np.abs(p.N0).max()
    Ms = p.eps_static * p.M_omega
    G = node_gradient(n)
    gcond = np.abs(G.T @ (Ms[:, None] * got.T)).max() / (np.abs(Ms[:, None] * got.T).max())
    assert gcond <= 1e-10, gcond
    A = p.K + sp.diags(Ms)
    f = A @ ref.T
    assert np.abs(A @ got.T - f).max() <= 1e-10 * np.abs(f).max()
    assert 0 < solver.iters[0] < 20000 and 0 < solver.iters[1] < 20000
