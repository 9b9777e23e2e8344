"""GPU parity of mrom_sweep_vjp (adjoint of Eqs. (17)-(19) in omega, s_sigma, s_mu) and of the
torch.autograd wrapper, against the oracle's dense tangents and central finite differences."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# the stated FP64 tolerance: relative 1e-10 (per (object, omega) against max |g_omega| of the
# object; a sum over frequencies against the sum of its terms' magnitudes)
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


@pytest.mark.parametrize("lu", [False, True], ids=["pencil", "lu"])
def test_vjp_matches_oracle_tangents(mrom, lu):
    """Both routes: the adjoint in the eigenbasis of each object's pencil (default) and by LU."""
    import torch
    from oracle import grads
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    h.set_solver(lu=lu)
    rs = [5, 24, 61, 96]
    objs = [reduced_object(20230711, 500 + k, r) for k, r in enumerate(rs)]
    roms = [mrom.ReducedObject.from_workload(h, o, with_cert=False) for o in objs]
    n_w = 37
    wo = log_omegas(1e1, 1e8, n_w)
    ss = np.array([0.5, 1.0, 1.7, 2.0])
    sm = np.array([1.0, 4.0, 17.0, 64.0])
    rng = np.random.default_rng(3)
    gR = rng.standard_normal((4, n_w, 3, 3))
    gI = rng.standard_normal((4, n_w, 3, 3))
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g_w = torch.empty((4, n_w), dtype=torch.float64, device="cuda")
    g_s = torch.empty(4, dtype=torch.float64, device="cuda")
    g_m = torch.empty(4, dtype=torch.float64, device="cuda")
    R = torch.empty((4, n_w, 3, 3), dtype=torch.float64, device="cuda")
    I = torch.empty_like(R)
    mrom.mrom_sweep_vjp(h, roms, t(wo), n_w, t(gR), t(gI), g_w, g_ssigma=g_s, g_smu=g_m, s_sigma=t(ss), s_mu=t(sm),
                        R=R, I=I)
    h.synchronize()
    for k, obj in enumerate(objs):
        Rr, Ir = grads.forward(obj, wo, ss[k], sm[k])
        assert np.abs(R[k].cpu().numpy() - Rr).max() <= 1e-10 * np.abs(Rr).max()
        assert np.abs(I[k].cpu().numpy() - Ir).max() <= 1e-9 * np.abs(Ir).max()
        dR, dI = grads.tangents(obj, wo, ss[k], sm[k])
        # per-frequency contributions of L to each derivative (the oracle's dense tangents)
        contrib = np.einsum("twij,wij->tw", dR, gR[k]) + np.einsum("twij,wij->tw", dI, gI[k])
        gw = contrib[0]
        assert np.abs(g_w[k].cpu().numpy() - gw).max() <= TOL * np.abs(gw).max(), (obj.r,)
        # dL/ds is a sum over the frequencies: relative to the sum of its terms' magnitudes
        assert abs(g_s[k].item() - contrib[1].sum()) <= TOL * np.abs(contrib[1]).sum(), (obj.r,)
        assert abs(g_m[k].item() - contrib[2].sum()) <= TOL * np.abs(contrib[2]).sum(), (obj.r,)


@pytest.mark.parametrize("lu", [False, True], ids=["pencil", "lu"])
def test_vjp_scale_gradients_per_frequency(mrom, lu):
    """dL/ds_sigma and dL/ds_mu of one frequency at a time (n_w = 1), so that each is compared with
    the oracle's tangent at that frequency alone, relative to that frequency's term scale
    sum_ij |dR_ij/ds| |gR_ij| + |dI_ij/ds| |gI_ij|."""
    import torch
    from oracle import grads
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    h.set_solver(lu=lu)
    objs = [reduced_object(20230711, 520 + k, r) for k, r in enumerate([7, 33, 80])]
    roms = [mrom.ReducedObject.from_workload(h, o, with_cert=False) for o in objs]
    ss = np.array([0.6, 1.0, 1.9])
    sm = np.array([1.5, 8.0, 50.0])
    rng = np.random.default_rng(5)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    for w in log_omegas(1e1, 1e8, 9):
        gR = rng.standard_normal((3, 1, 3, 3))
        gI = rng.standard_normal((3, 1, 3, 3))
        g_w = torch.empty((3, 1), dtype=torch.float64, device="cuda")
        g_s = torch.empty(3, dtype=torch.float64, device="cuda")
        g_m = torch.empty(3, dtype=torch.float64, device="cuda")
        mrom.mrom_sweep_vjp(h, roms, t(np.array([w])), 1, t(gR), t(gI), g_w, g_ssigma=g_s, g_smu=g_m,
                            s_sigma=t(ss), s_mu=t(sm))
        h.synchronize()
        for k, obj in enumerate(objs):
            dR, dI = grads.tangents(obj, np.array([w]), ss[k], sm[k])
            contrib = np.einsum("twij,wij->t", dR, gR[k]) + np.einsum("twij,wij->t", dI, gI[k])
            sc = (np.abs(dR) * np.abs(gR[k])[None]).sum(axis=(1, 2, 3)) + \
                 (np.abs(dI) * np.abs(gI[k])[None]).sum(axis=(1, 2, 3))
            got = (g_w[k, 0].item(), g_s[k].item(), g_m[k].item())
            for j in range(3):
                assert abs(got[j] - contrib[j]) <= TOL * sc[j], (obj.r, w, j)


def test_autograd_matches_finite_differences(mrom):
    import torch
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    objs = [reduced_object(20230711, 700 + k, r) for k, r in enumerate([12, 40])]
    roms = [mrom.ReducedObject.from_workload(h, o, with_cert=False) for o in objs]
    wo = torch.as_tensor(log_omegas(1e2, 1e6, 9), device="cuda").requires_grad_(True)
    ss = torch.tensor([1.3, 0.8], dtype=torch.float64, device="cuda", requires_grad=True)
    sm = torch.tensor([2.0, 9.0], dtype=torch.float64, device="cuda", requires_grad=True)
    wR = torch.randn((2, 9, 3, 3), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    wI = torch.randn((2, 9, 3, 3), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))

    def loss(w, s1, s2):
        R, I = mrom.signature(h, roms, w, s1, s2)
        return (wR * R).sum() + (wI * I).sum()

    L = loss(wo, ss, sm)
    L.backward()

    def central(x, k, rel):
        hstep = rel * x[k].item()
        x[k] += hstep
        Lp = loss(wo, ss, sm).item()
        x[k] -= 2 * hstep
        Lm = loss(wo, ss, sm).item()
        x[k] += hstep
        return (Lp - Lm) / (2 * hstep)

    # L is a sum of +-terms of size ~1e6 whose rounding noise (~kappa(A) eps) limits a difference
    # quotient: h = 1e-4 (truncation ~1e-8) is checked tightly, h = 1e-6 (the configured step) at
    # the size of its noise.
    with torch.no_grad():
        for x, g in ((ss, ss.grad), (sm, sm.grad), (wo, wo.grad)):
            for k in ([0, 1] if x is not wo else [2, 6]):
                assert g[k].item() == pytest.approx(central(x, k, 1e-4), rel=1e-6)
                assert g[k].item() == pytest.approx(central(x, k, 1e-6), rel=1e-4)


def test_least_squares_fit_of_material_scales(mrom):
    """Fit (s_sigma, s_mu) of an object to a target signature made with scales drawn from the
    held-out seed 20230712, using gradients from the adjoint kernel."""
    import torch
    from scipy.optimize import minimize
    from workloads import log_omegas, reduced_object
    h = mrom.Handle(0)
    obj = reduced_object(20230711, 900, 30)
    rom = mrom.ReducedObject.from_workload(h, obj, with_cert=False)
    rng = np.random.default_rng(20230712)
    true_s = np.array([rng.uniform(0.5, 2.0), np.exp(rng.uniform(0.0, np.log(64.0)))])
    wo = torch.as_tensor(log_omegas(1e1, 1e8, 80), device="cuda")
    t1 = lambda v: torch.tensor([v], dtype=torch.float64, device="cuda")
    with torch.no_grad():
        Rt, It = mrom.signature(h, [rom], wo, t1(true_s[0]), t1(true_s[1]))
        sR, sI = Rt.abs().amax(dim=(2, 3), keepdim=True), It.abs().amax(dim=(2, 3), keepdim=True)

    def fun(x):
        a = torch.tensor([np.exp(x[0])], dtype=torch.float64, device="cuda", requires_grad=True)
        b = torch.tensor([np.exp(x[1])], dtype=torch.float64, device="cuda", requires_grad=True)
        R, I = mrom.signature(h, [rom], wo, a, b)
        L = (((R - Rt) / sR) ** 2).sum() + (((I - It) / sI) ** 2).sum()
        L.backward()
        return L.item(), np.array([a.grad.item() * a.item(), b.grad.item() * b.item()])

    res = minimize(fun, np.zeros(2), jac=True, method="L-BFGS-B", options={"maxiter": 200, "gtol": 1e-12, "ftol": 1e-16})
    fit = np.exp(res.x)
    assert np.allclose(fit, true_s, rtol=1e-5), (fit, true_s)


def test_vjp_routes_agree_with_regularisation_and_without_scales(mrom):
    """An object with Me = U^H (eps M) U (V^H Me V enters R and the adjoint source) and calls
    without s_mu / g_smu: the pencil route reproduces the LU route (itself pinned to the oracle)."""
    import torch
    from workloads import log_omegas, reduced_object
    obj = reduced_object(77, 3, 40)
    rng = np.random.default_rng(11)
    Z = (rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))) * 1e-3
    Me = Z @ Z.conj().T
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    n_w = 45
    wo = t(log_omegas(1e1, 1e8, n_w))
    gR = t(rng.standard_normal((1, n_w, 3, 3)))
    gI = t(rng.standard_normal((1, n_w, 3, 3)))
    out = []
    for lu in (False, True):
        h = mrom.Handle(0)
        h.set_solver(lu=lu)
        ro = mrom.ReducedObject(h, 40, t(obj.K), t(obj.C), t(obj.B), obj.c00, K_in=t(obj.K_in), Me=t(Me))
        res = []
        for scales in (True, False):
            g_w = torch.empty((1, n_w), dtype=torch.float64, device="cuda")
            g_s = torch.empty(1, dtype=torch.float64, device="cuda")
            g_m = torch.empty(1, dtype=torch.float64, device="cuda") if scales else None
            R = torch.empty((1, n_w, 3, 3), dtype=torch.float64, device="cuda")
            I = torch.empty_like(R)
            kw = dict(s_sigma=t(np.array([1.3])), s_mu=t(np.array([7.0]))) if scales else {}
            mrom.mrom_sweep_vjp(h, [ro], wo, n_w, gR, gI, g_w, g_ssigma=g_s, g_smu=g_m, R=R, I=I, **kw)
            h.synchronize()
            res.append([x.cpu().numpy() for x in (g_w, g_s, R, I)] + ([g_m.cpu().numpy()] if scales else []))
        out.append(res)
    for a, b in zip(out[0], out[1]):
        gw_p, gw_l = a[0], b[0]
        assert np.abs(gw_p - gw_l).max() <= TOL * np.abs(gw_l).max()
        assert np.allclose(a[1], b[1], rtol=TOL)
        assert np.abs(a[2] - b[2]).max() <= TOL * np.abs(b[2]).max()
        assert np.abs(a[3] - b[3]).max() <= 1e-9 * np.abs(b[3]).max()
        if len(a) > 4:
            assert np.allclose(a[4], b[4], rtol=TOL)
