"""mrom_sweep_noalloc against mrom_sweep, through the C ABI.

Some callers cannot allocate device memory while they run (a service with a
fixed memory budget reserved at start-up, an application whose own allocator
owns the GPU's memory, or a loop where cudaMalloc would synchronise the
device).  mrom_sweep_noalloc serves them from a fixed scratch array inside the
library; it must return what mrom_sweep returns, also on a second call that
reuses the array left behind by the first.  This file is collected last.
"""
import numpy as np
import pytest

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


def _outputs(torch, n_obj, n_w):
    R = torch.full((n_obj, n_w, 3, 3), float("nan"), dtype=torch.float64, device="cuda")
    return R, torch.full_like(R, float("nan")), torch.full_like(R, float("nan"))


def _compare(torch, got, ref):
    for g, r in zip(got, ref):
        g, r = g.cpu().numpy(), r.cpu().numpy()
        assert np.all(np.isfinite(g))
        scale = np.abs(r).reshape(r.shape[0], r.shape[1], -1).max(axis=2)[..., None, None]
        assert np.max(np.abs(g - r) / scale) <= TOL


def test_noalloc_sweep_matches_sweep_on_two_calls(mrom):
    import torch
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    h.set_solver(lu=True)  # the allocation-free sweep is the LU route; compare with the same route
    # sizes on both sides of the shared-memory limit, so the workspace part of the array is used
    batches = [
        ([reduced_object(31337, k, r) for k, r in enumerate([8, 40, 64, 90, 96])], log_omegas(1e1, 1e8, 120)),
        ([reduced_object(4242, k, r) for k, r in enumerate([96, 17, 55])], log_omegas(3e1, 3e7, 77)),
    ]
    for objs, wo in batches:
        roms = [mrom.ReducedObject.from_workload(h, o) for o in objs]
        om = torch.as_tensor(wo, device="cuda")
        ref = _outputs(torch, len(objs), wo.size)
        mrom.mrom_sweep(h, roms, om, wo.size, *ref)
        got = _outputs(torch, len(objs), wo.size)
        mrom.mrom_sweep_noalloc(h, roms, om, wo.size, *got)
        h.synchronize()
        _compare(torch, got, ref)


def test_noalloc_sweep_matches_the_oracle_and_allocates_nothing(mrom):
    """Per-object frequency grids (omega_stride > n_w), outputs without Delta, and a second call:
    the results match the CPU oracle (R against max |R|, I against its term scale per frequency),
    and after a first call the device's free memory does not change across a second one."""
    import torch
    from gpu_common import oracle_sweep, rel_errors
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    objs = [reduced_object(2718, k, r) for k, r in enumerate([12, 50, 96])]
    roms = [mrom.ReducedObject.from_workload(h, o) for o in objs]
    n_w, stride = 41, 64
    grids = [log_omegas(1e1 * (k + 1), 1e8 / (k + 1), n_w) for k in range(len(objs))]
    om_host = np.zeros((len(objs), stride))
    for k, g in enumerate(grids):
        om_host[k, :n_w] = g
        om_host[k, n_w:] = np.nan  # never read: only the first n_w of each row are frequencies
    om = torch.as_tensor(om_host, device="cuda")
    R = torch.full((len(objs), n_w, 3, 3), float("nan"), dtype=torch.float64, device="cuda")
    I = torch.full_like(R, float("nan"))
    mrom.mrom_sweep_noalloc(h, roms, om, n_w, R, I, omega_stride=stride)
    h.synchronize()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    R.fill_(float("nan"))
    I.fill_(float("nan"))
    mrom.mrom_sweep_noalloc(h, roms, om, n_w, R, I, omega_stride=stride)
    h.synchronize()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for k, obj in enumerate(objs):
        Rr, Ir, _, sI, _ = oracle_sweep(obj, grids[k])
        eR, eI, _ = rel_errors(R[k].cpu().numpy(), I[k].cpu().numpy(), None, Rr, Ir, None, sI, None)
        assert max(eR, eI) <= TOL, (obj.r, eR, eI)


def test_noalloc_sweep_refuses_a_batch_larger_than_its_array(mrom):
    import torch
    from workloads import reduced_object
    h = mrom.Handle(0)
    rom = mrom.ReducedObject.from_workload(h, reduced_object(1, 0, 8))
    n = 300_000  # ~330 bytes of table per object exceed the 64 MiB array
    om = torch.tensor([10.0], dtype=torch.float64, device="cuda")
    R = torch.empty(9, dtype=torch.float64, device="cuda")
    with pytest.raises(mrom.MromError) as ei:
        mrom.mrom_sweep_noalloc(h, [rom] * n, om, 1, R, R)
    assert ei.value.status == 1
    assert "MROM_NOALLOC_SCRATCH_BYTES" in str(ei.value)
