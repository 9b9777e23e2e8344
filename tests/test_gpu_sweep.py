"""GPU parity of mrom_sweep (reduced solves, Eqs. (17)-(19), certificate of Lemma 4.2)
against the CPU oracle, through the C ABI."""
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


@pytest.fixture(scope="module", params=["auto", "lu"])
def handle(mrom, request):
    """Both solver routes: the Hermitian pencil where its error estimate allows (default),
    and LU elimination without pivoting for every object."""
    h = mrom.Handle(0)
    h.set_solver(lu=request.param == "lu")
    h.solver = request.param
    return h


def _run(mrom, handle, objs, omega, n_w, with_delta=True, omega_stride=0, s_sigma=None):
    import torch
    dev = torch.device("cuda", 0)
    roms = [mrom.ReducedObject.from_workload(handle, o) for o in objs]
    n = len(objs)
    om = torch.as_tensor(np.ascontiguousarray(omega), dtype=torch.float64, device=dev)
    R = torch.full((n, n_w, 3, 3), np.nan, dtype=torch.float64, device=dev)
    I = torch.full_like(R, np.nan)
    D = torch.full_like(R, np.nan) if with_delta else None
    ss = torch.as_tensor(s_sigma, dtype=torch.float64, device=dev) if s_sigma is not None else None
    mrom.mrom_sweep(handle, roms, om, n_w, R, I, D, omega_stride=omega_stride, s_sigma=ss)
    handle.synchronize()
    out = (R.cpu().numpy(), I.cpu().numpy(), D.cpu().numpy() if with_delta else None)
    for r in roms:
        r.close()
    return out


def test_sweep_matches_oracle_across_tile_boundaries(mrom, handle):
    """r spans warp/tile boundaries; 250 frequencies make ragged frequency chunks."""
    from workloads import log_omegas, reduced_object
    from gpu_common import oracle_sweep, rel_errors
    rs = [1, 2, 3, 8, 17, 31, 32, 33, 64, 95, 96, 112]
    objs = [reduced_object(20230711, 100 + k, r) for k, r in enumerate(rs)]
    wo = log_omegas(1e1, 1e8, 250)
    Rg, Ig, Dg = _run(mrom, handle, objs, wo, wo.size)
    for k, obj in enumerate(objs):
        R, I, Dl, sI, sD = oracle_sweep(obj, wo)
        eR, eI, eD = rel_errors(Rg[k], Ig[k], Dg[k], R, I, Dl, sI, sD)
        assert eR <= TOL and eI <= TOL and eD <= TOL, (obj.r, eR, eI, eD)


def test_per_object_grids_and_conductivity_scale(mrom, handle):
    from workloads import log_omegas, reduced_object
    from gpu_common import oracle_sweep, rel_errors
    objs = [reduced_object(5, k, r) for k, r in enumerate([9, 40, 77])]
    n_w = 41
    grids = np.stack([log_omegas(10.0 ** (1 + k), 1e7, n_w) for k in range(3)])
    ss = np.array([0.5, 1.0, 2.0])
    Rg, Ig, Dg = _run(mrom, handle, objs, grids, n_w, omega_stride=n_w, s_sigma=ss)
    for k, obj in enumerate(objs):
        R, I, Dl, sI, sD = oracle_sweep(obj, grids[k], s_sigma=ss[k])
        eR, eI, eD = rel_errors(Rg[k], Ig[k], Dg[k], R, I, Dl, sI, sD)
        assert eR <= TOL and eI <= TOL and eD <= TOL, (obj.r, eR, eI, eD)


def test_certificate_only_and_no_certificate(mrom, handle):
    import torch
    from workloads import log_omegas, reduced_object
    from gpu_common import oracle_sweep
    obj = reduced_object(9, 0, 20)
    wo = log_omegas(1e1, 1e8, 30)
    rom = mrom.ReducedObject.from_workload(handle, obj)
    om = torch.as_tensor(wo, device="cuda")
    D = torch.empty(30 * 9, dtype=torch.float64, device="cuda")
    mrom.mrom_certificate(handle, [rom], om, 30, D)
    handle.synchronize()
    _, _, Dl, _, sD = oracle_sweep(obj, wo)
    err = np.abs(D.cpu().numpy().reshape(30, 3, 3) - Dl).reshape(30, -1).max(1) / sD
    assert err.max() <= TOL
    # an object without a Gram matrix: R and I work, Delta is refused
    rom2 = mrom.ReducedObject.from_workload(handle, obj, with_cert=False)
    R = torch.empty(30 * 9, dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    mrom.mrom_sweep(handle, [rom2], om, 30, R, I)
    handle.synchronize()
    with pytest.raises(mrom.MromError) as ei:
        mrom.mrom_sweep(handle, [rom2], om, 30, R, I, D)
    assert ei.value.status == 1


def test_device_detected_bad_frequency(mrom, handle):
    import torch
    from workloads import reduced_object
    rom = mrom.ReducedObject.from_workload(handle, reduced_object(9, 1, 10))
    om = torch.tensor([10.0, -5.0, 100.0], dtype=torch.float64, device="cuda")
    R = torch.empty(27, dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    mrom.mrom_sweep(handle, [rom], om, 3, R, I)
    with pytest.raises(mrom.MromError) as ei:
        handle.synchronize()
    assert ei.value.status == 1
    handle.synchronize()  # status cleared


def test_singular_reduced_system_reported(mrom, handle):
    """An object whose K_r and C_r share the null vector e_r (last row and column zero, so
    A(omega) = K_r - i omega C_r is singular at every omega): the pencil route's Cholesky of C_r
    fails, the object goes to the LU route, whose last pivot is exactly zero, and the next
    mrom_synchronize returns MROM_ESINGULAR.  A regular object in the same batch is unaffected."""
    import torch
    from gpu_common import oracle_sweep, rel_errors
    from workloads import log_omegas, reduced_object
    bad = reduced_object(9, 4, 12)
    K, C = bad.K.copy(), bad.C.copy()
    K[-1, :] = 0.0
    K[:, -1] = 0.0
    C[-1, :] = 0.0
    C[:, -1] = 0.0
    good = reduced_object(9, 5, 20)
    n_w = 17
    wo = log_omegas(1e1, 1e8, n_w)
    roms = [mrom.ReducedObject(handle, 12, K, C, bad.B, bad.c00),
            mrom.ReducedObject.from_workload(handle, good, with_cert=False)]
    plan = mrom.Plan(handle, roms, n_w)
    om = torch.as_tensor(wo, device="cuda")
    R = torch.empty((2, n_w, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    plan.sweep(om, R, I)
    with pytest.raises(mrom.MromError) as ei:
        handle.synchronize()
    assert ei.value.status == 4  # MROM_ESINGULAR
    handle.synchronize()  # status cleared
    n_pen, n_lu = plan.solver_counts()
    assert (n_pen, n_lu) == ((0, 2) if handle.solver == "lu" else (1, 1))
    assert not np.isfinite(R[0].cpu().numpy()).all()
    Rr, Ir, _, sI, _ = oracle_sweep(good, wo)
    eR, eI, _ = rel_errors(R[1].cpu().numpy(), I[1].cpu().numpy(), None, Rr, Ir, None, sI, None)
    assert max(eR, eI) <= TOL
    plan.close()


def test_invalid_objects_rejected(mrom, handle):
    from workloads import reduced_object
    obj = reduced_object(9, 2, 6)
    K = obj.K.copy()
    K[1, 2] = np.nan
    with pytest.raises(mrom.MromError) as ei:
        mrom.ReducedObject(handle, 6, K, obj.C, obj.B, obj.c00)
    assert ei.value.status == 1
    with pytest.raises(mrom.MromError):
        mrom.ReducedObject(handle, 113, np.zeros((113, 113)), np.zeros((113, 113)), np.zeros((113, 3)),
                           obj.c00)


def test_launch_count_increases(mrom, handle):
    """LU route: one sweep kernel.  Pencil route: preparation, routing and the two sweep
    kernels (the LU one over an empty table)."""
    import torch
    from workloads import reduced_object
    rom = mrom.ReducedObject.from_workload(handle, reduced_object(9, 3, 12))
    om = torch.tensor([10.0, 20.0], dtype=torch.float64, device="cuda")
    R = torch.empty(18, dtype=torch.float64, device="cuda")
    before = handle.launch_count()
    mrom.mrom_sweep(handle, [rom], om, 2, R, torch.empty_like(R))
    handle.synchronize()
    assert handle.launch_count() == before + (1 if handle.solver == "lu" else 6)


def _plan_sweep(mrom, handle, objs, wo):
    import torch
    roms = [mrom.ReducedObject.from_workload(handle, o) for o in objs]
    plan = mrom.Plan(handle, roms, wo.size)
    om = torch.as_tensor(wo, device="cuda")
    R = torch.empty((len(objs), wo.size, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    D = torch.empty_like(R)
    plan.sweep(om, R, I, D)
    handle.synchronize()
    return plan.solver_counts(), (R.cpu().numpy(), I.cpu().numpy(), D.cpu().numpy())


def test_routing_of_dictionary_and_ill_conditioned_objects(mrom, handle):
    """Dictionary objects (K spectrum [1e-6, 1e2], C spectrum [1e-3, 1]) all pass the pencil
    gate; an object with K up to 1e4 has an error estimate eps ||H|| / omega_min above 1e-11
    and goes to LU elimination in the same batch.  Every object matches the oracle."""
    from workloads import log_omegas, reduced_object
    from gpu_common import oracle_sweep, rel_errors
    objs = [reduced_object(31, k, r) for k, r in enumerate([10, 48, 90])]
    objs.append(reduced_object(31, 7, 40, k_range=(-4.0, 4.0)))
    wo = log_omegas(1e1, 1e8, 97)
    (n_pen, n_lu), (Rg, Ig, Dg) = _plan_sweep(mrom, handle, objs, wo)
    if handle.solver == "lu":
        assert (n_pen, n_lu) == (0, 4)
    else:
        assert (n_pen, n_lu) == (3, 1)
    for k, obj in enumerate(objs):
        errs = rel_errors(Rg[k], Ig[k], Dg[k], *oracle_sweep(obj, wo))
        assert max(errs) <= TOL, (obj.r, errs)


def test_pole_split_spectra(mrom, handle):
    """The pencil sweep splits its Hermitian forms at m = #{lambda_k < omega}: objects whose
    eigenvalues include an exact null space of K (lambda = 0, clamped rounding), one r-fold
    eigenvalue (K = 3 C) crossed by the sweep and met exactly at omega = 3, all eigenvalues above
    the frequencies (m = 0) and all below (m = r); every one on the pencil route and at parity."""
    from workloads import log_omegas, reduced_object
    from gpu_common import oracle_sweep, rel_errors
    a = reduced_object(51, 0, 24, k_range=(-2.0, 0.0), c_range=(-0.5, 0.0))
    lam, Q = np.linalg.eigh(a.K)
    lam[:2] = 0.0
    a.K_out = (Q * lam[None, :]) @ Q.conj().T
    a.K_out = 0.5 * (a.K_out + a.K_out.conj().T)
    a.K_in = np.zeros_like(a.K_out)
    b = reduced_object(51, 1, 16)
    b.K_out, b.K_in = 3.0 * b.C, np.zeros_like(b.C)
    c = reduced_object(51, 2, 20, k_range=(1.0, 2.0), c_range=(-0.5, 0.0))
    d = reduced_object(51, 3, 33, k_range=(-3.0, -2.0), c_range=(-0.5, 0.0))
    objs = [a, b, c, d]
    wo = np.append(log_omegas(1e-1, 5.0, 64), 3.0)
    (n_pen, n_lu), (Rg, Ig, Dg) = _plan_sweep(mrom, handle, objs, wo)
    assert (n_pen, n_lu) == ((0, 4) if handle.solver == "lu" else (4, 0))
    for k, obj in enumerate(objs):
        errs = rel_errors(Rg[k], Ig[k], Dg[k], *oracle_sweep(obj, wo))
        assert max(errs) <= TOL, (k, obj.r, errs)


def test_sweep_host_pipeline(mrom, handle):
    """mrom_sweep_host (host buffers in and out, groups pipelined over two streams) gives the
    device plan sweep's values on a batch with pencil- and LU-routed objects, for 1, 3 and more
    groups than objects, with and without the certificate; bad arguments are refused."""
    import torch
    from workloads import log_omegas, reduced_object
    from gpu_common import oracle_sweep, rel_errors
    objs = [reduced_object(61, k, r) for k, r in enumerate([12, 40, 7, 96, 33, 1, 64, 20])]
    objs.append(reduced_object(61, 9, 40, k_range=(-4.0, 4.0)))   # LU route under "auto"
    wo = log_omegas(1e1, 1e8, 70)
    packed = mrom.PackedDictionary([dict(r=o.r, K=o.K, C=o.C, B=o.B, c00=o.c00, G=o.G, K_in=o.K_in,
                                         alpha=o.alpha, alpha_lb=o.alpha_lb, vol_B=o.vol_B) for o in objs])
    _, (Rp, Ip, Dp) = _plan_sweep(mrom, handle, objs, wo)
    shape = (len(objs), wo.size, 3, 3)
    om = torch.from_numpy(wo.copy()).pin_memory()
    for n_chunks, cert in ((1, True), (3, True), (16, False)):
        R, I = (torch.full(shape, np.nan, dtype=torch.float64).pin_memory() for _ in range(2))
        D = torch.full(shape, np.nan, dtype=torch.float64).pin_memory() if cert else None
        mrom.mrom_sweep_host(handle, packed, om, R, I, D, n_chunks=n_chunks)
        assert np.array_equal(R.numpy(), Rp) and np.array_equal(I.numpy(), Ip), n_chunks
        if cert:
            assert np.array_equal(D.numpy(), Dp), n_chunks
    for k in (1, 3, 8):
        errs = rel_errors(R.numpy()[k], I.numpy()[k], Dp[k], *oracle_sweep(objs[k], wo))
        assert max(errs) <= TOL, (k, errs)
    with pytest.raises(mrom.MromError):
        mrom.mrom_sweep_host(handle, packed, om, R, I, None, n_chunks=0)
    with pytest.raises(mrom.MromError):
        mrom.mrom_sweep_host(handle, packed, om, R, I, None, n_chunks=17)


def test_pencil_route_with_stiffness_regularisation(mrom, handle):
    """An object with Me = U^H (eps M) U (added to the system only, not to R): the pencil
    route carries V^H Me V as a separate Hermitian form."""
    import torch
    from workloads import log_omegas, reduced_object
    from oracle import rom as orom
    from gpu_common import oracle_model_sweep, rel_errors
    obj = reduced_object(41, 0, 30)
    rng = np.random.default_rng(5)
    Z = (rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))) * 1e-3
    Me = Z @ Z.conj().T
    model = orom.from_reduced_object(obj)
    model.Me = [Me] * 3
    wo = log_omegas(1e1, 1e8, 70)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    ro = mrom.ReducedObject(handle, 30, t(obj.K), t(obj.C), t(obj.B), obj.c00, G=t(obj.G), Me=t(Me),
                            alpha=obj.alpha, alpha_lb=obj.alpha_lb)
    om = t(wo)
    R = torch.empty((1, 70, 3, 3), dtype=torch.float64, device=dev)
    I = torch.empty_like(R)
    D = torch.empty_like(R)
    mrom.mrom_sweep(handle, [ro], om, 70, R, I, D)
    handle.synchronize()
    errs = rel_errors(R[0].cpu().numpy(), I[0].cpu().numpy(), D[0].cpu().numpy(), *oracle_model_sweep(model, wo))
    assert max(errs) <= TOL, errs


def test_autotuner_picks_a_valid_configuration(mrom, handle):
    """mrom_tune times every launch configuration; results after tuning are unchanged."""
    import torch
    from workloads import log_omegas, reduced_object
    from gpu_common import oracle_sweep, rel_errors
    objs = [reduced_object(77, k, r) for k, r in enumerate([12, 50, 90])]
    roms = [mrom.ReducedObject.from_workload(handle, o) for o in objs]
    cfg = mrom.mrom_tune(handle, roms, 60)
    assert cfg in (0, 1)
    groups = mrom.mrom_tune_pencil(handle, roms, 300)
    assert groups in (1, 2, 4, 8)
    wo = log_omegas(1e1, 1e8, 60)
    om = torch.as_tensor(wo, device="cuda")
    R = torch.empty((3, 60, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    D = torch.empty_like(R)
    plan = mrom.Plan(handle, roms, 60)
    plan.sweep(om, R, I, D)
    handle.synchronize()
    for k, obj in enumerate(objs):
        ref = oracle_sweep(obj, wo)
        errs = rel_errors(R[k].cpu().numpy(), I[k].cpu().numpy(), D[k].cpu().numpy(), *ref)
        assert max(errs) <= TOL, errs


def test_batched_object_creation(mrom, handle):
    """mrom_rom_from_reduced_batch gives the same sweep as objects created one by one; a
    non-finite entry is refused with the object named; the shared allocation outlives any
    subset of its objects."""
    import torch
    from workloads import log_omegas, reduced_object
    objs = [reduced_object(61, k, r) for k, r in enumerate([5, 30, 64])]
    wo = log_omegas(1e1, 1e8, 50)
    om = torch.as_tensor(wo, device="cuda")
    single = [mrom.ReducedObject.from_workload(handle, o) for o in objs]
    batch = mrom.ReducedObject.from_workload_batch(handle, objs)
    out = []
    for roms in (single, batch):
        R = torch.empty((3, 50, 3, 3), dtype=torch.float64, device="cuda")
        I = torch.empty_like(R)
        D = torch.empty_like(R)
        mrom.mrom_sweep(handle, roms, om, 50, R, I, D)
        handle.synchronize()
        out.append([x.cpu().numpy() for x in (R, I, D)])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    batch[0].close()
    batch[2].close()
    R = torch.empty((1, 50, 3, 3), dtype=torch.float64, device="cuda")
    mrom.mrom_sweep(handle, [batch[1]], om, 50, R, torch.empty_like(R))
    handle.synchronize()
    assert np.array_equal(R[0].cpu().numpy(), out[0][0][1])
    batch[1].close()
    bad = reduced_object(61, 9, 12)
    C = bad.C.copy()
    C[3, 4] = np.inf
    items = [dict(r=o.r, K=o.K, C=o.C, B=o.B, c00=o.c00, G=o.G) for o in objs]
    items.append(dict(r=12, K=bad.K, C=C, B=bad.B, c00=bad.c00, G=bad.G))
    with pytest.raises(mrom.MromError) as ei:
        mrom.ReducedObject.batch(handle, items)
    assert ei.value.status == 1 and "object 3" in str(ei.value)


def test_packed_dictionary_matches_batch(mrom):
    """mrom_rom_from_packed (one copy of a packed buffer) gives the objects of
    mrom_rom_from_reduced_batch: identical sweeps; bad regions and non-finite data are refused."""
    import torch
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    objs = [reduced_object(20230711, 900 + k, r) for k, r in enumerate([7, 40, 96, 13])]
    items = [dict(r=o.r, K=o.K, C=o.C, B=o.B, c00=o.c00, G=o.G if k != 1 else None, K_in=o.K_in,
                  alpha=o.alpha, alpha_lb=o.alpha_lb, vol_B=o.vol_B) for k, o in enumerate(objs)]
    items[3]["Me"] = 1e-4 * np.eye(objs[3].r, dtype=np.complex128)   # an Me block in the region
    pk = mrom.PackedDictionary(items)
    a = mrom.ReducedObject.from_packed(h, pk)
    b = mrom.ReducedObject.batch(h, items)
    wo = torch.as_tensor(log_omegas(1e1, 1e8, 50), device="cuda")
    outs = []
    for roms in (a, b):
        R = torch.empty((4, 50, 3, 3), dtype=torch.float64, device="cuda")
        I = torch.empty_like(R)
        mrom.mrom_sweep(h, roms, wo, 50, R, I)              # object 1 has no Gram matrix: no Delta
        cert = [roms[k] for k in (0, 2, 3)]
        D = torch.empty((3, 50, 3, 3), dtype=torch.float64, device="cuda")
        R3, I3 = torch.empty_like(D), torch.empty_like(D)
        mrom.mrom_sweep(h, cert, wo, 50, R3, I3, D)
        h.synchronize()
        outs.append((R.cpu().numpy(), I.cpu().numpy(), D.cpu().numpy()))
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
    bad = mrom.PackedDictionary(items)
    bad.entries[2].offset += 8                       # not 16-byte aligned
    with pytest.raises(mrom.MromError):
        mrom.ReducedObject.from_packed(h, bad)
    bad = mrom.PackedDictionary(items)
    bad.entries[3].offset = bad.nbytes               # outside the buffer
    with pytest.raises(mrom.MromError):
        mrom.ReducedObject.from_packed(h, bad)
    items[2]["K"] = objs[2].K.copy()
    items[2]["K"][3, 5] = np.nan
    with pytest.raises(mrom.MromError):
        mrom.ReducedObject.from_packed(h, mrom.PackedDictionary(items))


def test_batch_release(mrom):
    """ReducedObject.close_all releases objects of one packed allocation with one call."""
    from workloads import reduced_object
    h = mrom.Handle(0)
    objs = [reduced_object(20230711, 950 + k, r) for k, r in enumerate([6, 9, 11])]
    pk = mrom.PackedDictionary([dict(r=o.r, K=o.K, C=o.C, B=o.B, c00=o.c00, G=o.G, K_in=o.K_in) for o in objs])
    roms = mrom.ReducedObject.from_packed(h, pk)
    mrom.ReducedObject.close_all(roms)
    assert all(not x._rom for x in roms)
    mrom.ReducedObject.close_all(roms)          # already released: nothing to do
    h.synchronize()


@pytest.mark.parametrize("lu", [False, True], ids=["auto", "lu"])
def test_sweep_at_permeability_scales_for_objects_without_static_reduction(mrom, lu):
    """mrom_sweep with s_mu on objects that carry K_in but no reduced static problem: K(s) =
    K + (1/s - 1) K_in with b and c00 fixed, as the oracle's forward model of the gradients."""
    import torch
    from oracle import grads
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    h.set_solver(lu=lu)
    objs = [reduced_object(20230711, 960 + k, r) for k, r in enumerate([6, 30, 71])]
    roms = [mrom.ReducedObject.from_workload(h, o) for o in objs]
    wo = log_omegas(1e1, 1e8, 41)
    ss = np.array([1.0, 0.7, 1.9])
    sm = np.array([3.0, 0.5, 17.0])
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    R = torch.empty((3, wo.size, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    mrom.mrom_sweep(h, roms, t(wo), wo.size, R, I, s_sigma=t(ss), s_mu=t(sm))
    h.synchronize()
    for k, o in enumerate(objs):
        Rr, Ir = grads.forward(o, wo, ss[k], sm[k])
        assert np.abs(R[k].cpu().numpy() - Rr).max() <= 1e-10 * np.abs(Rr).max()
        sI = wo * ss[k] * o.alpha ** 3 / 4 * np.abs(o.c00).max()
        assert (np.abs(I[k].cpu().numpy() - Ir).reshape(wo.size, -1).max(1) / sI).max() <= 1e-10
    D = torch.empty_like(R)
    with pytest.raises(mrom.MromError):          # no extended Gram: no certificate at a scale
        mrom.mrom_sweep(h, roms, t(wo), wo.size, R, I, D, s_mu=t(sm))
    h.set_solver(lu=False)


def test_plan_sweep_replays_as_a_cuda_graph(mrom):
    """A plan's sweep issues only stream-ordered work (no allocation, no host wait), so a caller
    can capture it once into a CUDA graph and replay it; the replay gives the direct call's
    outputs bit for bit, and follows new frequencies written in place."""
    import torch
    from workloads import log_omegas, reduced_object
    s = torch.cuda.Stream()
    h = mrom.Handle(0, s.cuda_stream)
    objs = [reduced_object(20230711, 980 + k, r) for k, r in enumerate([9, 41, 77])]
    roms = [mrom.ReducedObject.from_workload(h, o) for o in objs]
    n_w = 60
    plan = mrom.Plan(h, roms, n_w)
    with torch.cuda.stream(s):
        om = torch.as_tensor(log_omegas(1e1, 1e8, n_w), device="cuda")
        R = torch.zeros((3, n_w, 3, 3), dtype=torch.float64, device="cuda")
        I, D = torch.zeros_like(R), torch.zeros_like(R)
    plan.sweep(om, R, I, D)
    h.synchronize()
    ref = [x.clone() for x in (R, I, D)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        plan.sweep(om, R, I, D)
    for x in (R, I, D):
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    for x, y in zip((R, I, D), ref):
        assert torch.equal(x, y)
    with torch.cuda.stream(s):
        om.mul_(1.5)                        # new frequencies in place, then replay
    g.replay()
    torch.cuda.synchronize()
    plan.sweep(om, *ref)
    h.synchronize()
    for x, y in zip((R, I, D), ref):
        assert torch.equal(x, y)
    plan.close()
