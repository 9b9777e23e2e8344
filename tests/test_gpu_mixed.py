"""GPU parity of mrom_sweep_mixed (complex64 elimination + float64 refinement) against the
float64 oracle: 1e-5 with one refinement step (the mixed-precision target), 1e-9 with two."""
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


@pytest.mark.parametrize("n_refine,tol", [(1, 1e-5), (2, 1e-9)])
def test_mixed_sweep_matches_oracle(mrom, n_refine, tol):
    import torch
    from workloads import log_omegas, reduced_object
    from gpu_common import oracle_sweep, rel_errors
    h = mrom.Handle(0)
    rs = [1, 8, 17, 32, 33, 64, 95, 96]
    objs = [reduced_object(20230711, 300 + k, r) for k, r in enumerate(rs)]
    roms = [mrom.ReducedObject.from_workload(h, o) for o in objs]
    wo = log_omegas(1e1, 1e8, 150)
    om = torch.as_tensor(wo, device="cuda")
    R = torch.full((len(objs), wo.size, 3, 3), np.nan, dtype=torch.float64, device="cuda")
    I = torch.full_like(R, np.nan)
    D = torch.full_like(R, np.nan)
    mrom.mrom_sweep_mixed(h, roms, om, wo.size, R, I, D, n_refine=n_refine)
    h.synchronize()
    worst = 0.0
    for k, obj in enumerate(objs):
        errs = rel_errors(R[k].cpu().numpy(), I[k].cpu().numpy(), D[k].cpu().numpy(), *oracle_sweep(obj, wo))
        worst = max(worst, max(errs))
    assert worst <= tol, worst
