"""GPU tests of the boundary entry points added around the hot path:
``fill_set_spectrum`` (band-power updates without a new plan),
``fill_realize_batch`` (many plans in one call), non-finite data
(``FILL_EINVAL`` with the plan left usable) and the ``torch.autograd.Function``
``FillRealize`` (gradients for the data map and the band amplitudes through
``fill_backward``).
"""
import math

import numpy as np
import pytest

import oracle as O
from workloads import synth, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1109_0286_gb300 as cg  # noqa: E402

DT = {"fp64": torch.float64, "mixed": torch.float64, "fp32": torch.float32}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def band_case(n, nbands=32, band_frac=0.15, ndiscs=8, seed=14):
    k_lo = 2 * math.pi / n
    bidx, sig, noise = synth.band_templates_half(n, n, k_lo, nbands)
    obs = synth.mask_band_discs(n, n, int(round(band_frac * n)), ndiscs, 2.0, 12.0, seed)
    return bidx, sig, noise, obs


# ------------------------------------------------------------------ fill_set_spectrum

@pytest.mark.parametrize("mode", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("ny,nx", [(128, 128), (60, 140)])
def test_set_spectrum_equals_fresh_plan(mode, ny, nx):
    """A plan whose spectrum was replaced gives, bit for bit, what a plan
    built with the new spectrum gives (realization and operators), on a
    power-of-two and a mixed-radix grid."""
    P1 = synth.spectrum_cmb_like(ny, nx, 2 * math.pi / max(ny, nx))
    P2 = synth.spectrum_lorentz_beam(ny, nx, k0=2 * math.pi / 20, sb=1.2)
    obs = synth.mask_band_discs(ny, nx, ny // 8, 4, 2.0, 6.0, 5)
    d = torch.from_numpy(O.draw(O.hermitian_full(P2, nx), 3)).to(DT[mode]).cuda()
    tol = 1e-6 if mode == "fp32" else 1e-10
    a = cg.Plan(P1, obs, mode=mode, batch=2)
    a.realize(d, [1, 2], tol)                 # use it with the old spectrum first
    a.set_spectrum(P2)
    xa, sa = a.realize(d, [4, 5], tol)
    b = cg.Plan(P2, obs, mode=mode, batch=2)
    xb, sb = b.realize(d, [4, 5], tol)
    assert torch.equal(xa, xb)
    assert [s["iters"] for s in sa] == [s["iters"] for s in sb]
    x = torch.from_numpy(np.random.default_rng(1).standard_normal((ny, nx))).to(DT[mode]).cuda()
    for which in range(4):
        assert torch.equal(a.apply(which, x), b.apply(which, x)), which


def test_set_spectrum_rejects_invalid_and_keeps_the_plan():
    n = 64
    P, obs, _ = workload("plain64")
    plan = cg.Plan(P, obs, mode="fp64")
    d = torch.from_numpy(O.draw(O.hermitian_full(P, n), 1)).cuda()
    x0, _ = plan.realize(d, [2], 1e-10)
    bad = P.copy()
    bad[3, 5] = -1.0
    with pytest.raises(cg.FillError) as e:
        plan.set_spectrum(bad)
    assert e.value.status == 1 and "finite" in str(e.value)
    bad = P.copy()
    bad[1, 0] *= 1.5          # P(0, ky) != P(0, -ky)
    with pytest.raises(cg.FillError):
        plan.set_spectrum(bad)
    x1, _ = plan.realize(d, [2], 1e-10)
    assert torch.equal(x0, x1)


# ------------------------------------------------------------------ non-finite data

@pytest.mark.parametrize("mode", ["fp64", "mixed", "fp32"])
def test_nonfinite_data_is_einval_and_plan_stays_usable(mode):
    """NaN or Inf on an observed pixel: the realization's status is
    FILL_EINVAL, the call returns at once (no CG iteration), and a following
    valid call gives what a fresh plan gives.  NaN on a masked pixel is
    ignored (the values there are not data)."""
    P, obs, spec = workload("plain64")
    n = obs.shape[0]
    d0 = O.draw(O.hermitian_full(P, n), spec["data_seed"])
    tol = 1e-6 if mode == "fp32" else 1e-10
    plan = cg.Plan(P, obs, mode=mode, batch=2)
    iu = np.argwhere(obs == 1)[100]
    im = np.argwhere(obs == 0)[10]
    for bad in (np.nan, np.inf):
        d = d0.copy()
        d[tuple(iu)] = bad
        x, st = plan.realize(torch.from_numpy(d).to(DT[mode]).cuda(), [3, 4], tol, check=False)
        assert [s["status"] for s in st] == [1, 1]
        assert all(s["iters"] == 0 for s in st)
        with pytest.raises(cg.FillError) as e:
            plan.realize(torch.from_numpy(d).to(DT[mode]).cuda(), [3, 4], tol)
        assert e.value.status == 1
    dg = torch.from_numpy(d0).to(DT[mode]).cuda()
    x1, s1 = plan.realize(dg, [3, 4], tol)
    fresh = cg.Plan(P, obs, mode=mode, batch=2)
    x2, _ = fresh.realize(dg, [3, 4], tol)
    assert torch.equal(x1, x2) and all(s["status"] == 0 for s in s1)
    dm = d0.copy()
    dm[tuple(im)] = np.nan
    x3, s3 = plan.realize(torch.from_numpy(dm).to(DT[mode]).cuda(), [3, 4], tol)
    assert all(s["status"] == 0 for s in s3)
    assert torch.equal(x3, x1)


def test_nonfinite_one_map_of_a_batch():
    """Per-realization status: one bad map of a batch does not stop the
    others, and the call reports FILL_EINVAL."""
    P, obs, spec = workload("plain64")
    n = obs.shape[0]
    d0 = O.draw(O.hermitian_full(P, n), spec["data_seed"])
    ds = np.stack([d0, d0, d0])
    ds[1][obs == 1] = np.inf
    plan = cg.Plan(P, obs, mode="fp64", batch=3)
    x, st = plan.realize(torch.from_numpy(ds).cuda(), [5, 6, 7], 1e-10, check=False)
    assert [s["status"] for s in st] == [0, 1, 0]
    single = cg.Plan(P, obs, mode="fp64")
    for i in (0, 2):
        xi, _ = single.realize(torch.from_numpy(d0).cuda(), [5 + i], 1e-10)
        assert torch.equal(x[i], xi[0])


# ------------------------------------------------------------------ fill_realize_batch

@pytest.mark.parametrize("mode", ["fp32", "fp64", "mixed"])
def test_realize_batch_equals_single_plans(mode):
    """Plans with their own masks, spectra and grids (power-of-two and
    mixed-radix) in one fill_realize_batch call give what fill_realize gives
    each of them; a second call reuses the cached group."""
    shapes = [(64, 64, 1), (128, 128, 2), (64, 64, 1), (60, 140, 1)]
    plans, ds, seeds = [], [], []
    for k, (ny, nx, b) in enumerate(shapes):
        P = synth.spectrum_cmb_like(ny, nx, 2 * math.pi / 128)
        obs = synth.mask_area_target(ny, nx, seed=40 + k) if ny == nx else \
            synth.mask_band_discs(ny, nx, 6, 5, 2.0, 5.0, 40 + k)
        plans.append(cg.Plan(P, obs, mode=mode, batch=b))
        ds.append(torch.from_numpy(O.draw(O.hermitian_full(P, nx), 70 + k)).to(DT[mode]).cuda())
        seeds += [100 + 10 * k + i for i in range(b)]
    tol = 1e-6 if mode == "fp32" else 1e-10
    for rep in range(2):
        outs, stats = cg.realize_batch(plans, ds, seeds, tol)
        assert len(stats) == sum(p.batch for p in plans)
        assert all(s["status"] == 0 for s in stats)
        first = 0
        for p, d, o in zip(plans, ds, outs):
            x, _ = p.realize(d, seeds[first:first + p.batch], tol)
            assert torch.equal(o, x), (rep, first)
            first += p.batch


def test_group_with_mixed_radix_class_matches_oracle():
    """A group holding a mixed-radix size class (7000 x 600 maps scaled to
    140 x 60 and 350 x 120) next to a power-of-two class; the mixed-radix
    realizations against the oracle."""
    items = []
    for k, (ny, nx) in enumerate([(60, 140), (120, 350), (64, 64)]):
        P = synth.spectrum_cmb_like(ny, nx, 2 * math.pi / 512)
        obs = synth.mask_band_discs(ny, nx, 0, 12, 2.0, 6.7, 90 + k)
        items.append((P, obs, O.draw(O.hermitian_full(P, nx), 80 + k)))
    plans = [cg.Plan(P, obs, mode="fp64") for P, obs, _ in items]
    ds = [torch.from_numpy(d).cuda() for _, _, d in items]
    g = cg.Group(plans)
    outs, stats = g.realize(ds, [11, 12, 13], 1e-12)
    assert all(s["status"] == 0 for s in stats)
    for (P, obs, d), o, s in zip(items, outs, [11, 12, 13]):
        ref = O.realize(P, obs, d, s, tol=1e-13)
        m = obs == 0
        x = o[0].cpu().numpy()
        assert np.array_equal(x[~m], d[~m])
        assert rel(x[m], ref.x[m]) <= 1e-10


# ------------------------------------------------------------------ autograd

def _autograd_setup(n, mode, batch=1, nbands=32):
    bidx, sig, noise, obs = band_case(n, nbands=nbands)
    model = cg.BandPowerSpectrum(bidx, sig, noise)
    plan = cg.Plan(model(np.ones(nbands)), obs, mode=mode, backward=True, batch=batch)
    return model, plan, obs


@pytest.mark.parametrize("n,mode", [(128, "fp64"), (128, "mixed"), (2048, "fp32")])
def test_autograd_equals_plan_backward(n, mode):
    """loss.backward() through FillRealize gives, bit for bit, what
    Plan.backward gives for the same realization and dL/dx (at 2048^2 the
    differentiation workload's size: FP32 operator, tol 1e-6)."""
    nb = 32
    model, plan, obs = _autograd_setup(n, mode)
    P = model(np.ones(nb))
    tol = 1e-6 if mode == "fp32" else 1e-11
    d_np = O.draw(O.hermitian_full(P, n), 6)
    d = torch.from_numpy(d_np).to(DT[mode]).cuda().requires_grad_(True)
    a = torch.ones(nb, dtype=torch.float64, requires_grad=True)
    m = torch.from_numpy(obs == 0).cuda()
    x = cg.FillRealize.apply(d, a, plan, model, [7], tol)
    loss = (x[0] * x[0] * m).sum()
    loss.backward()
    # the same through the plan directly
    other = cg.Plan(P, obs, mode=mode, backward=True)
    other.set_bands(model.band_of_k, model.sig_half)
    x2, _ = other.realize(d.detach(), [7], tol)
    assert torch.equal(x.detach(), x2)
    g = (2.0 * x2 * m).contiguous()
    gd, gb, _ = other.backward(d.detach(), g, tol)
    assert torch.equal(d.grad, gd[0])
    assert np.array_equal(a.grad.numpy(), gb[0])


def test_autograd_matches_oracle_gradient():
    """The band and data gradients through FillRealize against the oracle's
    adjoint gradient (FP64 mode, both converged tightly)."""
    n, nb = 128, 32
    model, plan, obs = _autograd_setup(n, "fp64")
    P = model(np.ones(nb))
    d_np = O.draw(O.hermitian_full(P, n), 6)
    d = torch.from_numpy(d_np).cuda().requires_grad_(True)
    a = torch.ones(nb, dtype=torch.float64, requires_grad=True)
    m = torch.from_numpy(obs == 0).cuda()
    x = cg.FillRealize.apply(d, a, plan, model, [7], 1e-12)
    (x[0] * x[0] * m).sum().backward()
    real = O.realize(P, obs, d_np, 7, tol=1e-13)
    gd_o, gb_o, _ = O.backward(P, obs, d_np, 7, real, model.band_of_k, model.sig_half, tol=1e-13)
    u = obs == 1
    assert rel(d.grad.cpu().numpy()[u], gd_o[u]) <= 1e-8
    assert rel(a.grad.numpy(), gb_o) <= 1e-8


def test_autograd_finite_differences_with_one_plan():
    """Central differences (step 1e-4) of the loss in the band amplitudes,
    every evaluation through FillRealize on ONE plan (fill_set_spectrum per
    point, no new plan), against the autograd gradient at a != 1."""
    n, nb = 64, 16
    model, plan, obs = _autograd_setup(n, "fp64", nbands=nb)
    a0 = np.linspace(0.8, 1.3, nb)
    d_np = O.draw(O.hermitian_full(model(a0), n), 6)
    d = torch.from_numpy(d_np).cuda()
    m = torch.from_numpy(obs == 0).cuda()

    def loss(a_np, grad=False):
        a = torch.from_numpy(np.array(a_np)).requires_grad_(grad)
        x = cg.FillRealize.apply(d, a, plan, model, [5], 1e-13)
        L = (x[0] * x[0] * m).sum()
        if grad:
            L.backward()
            return float(L.detach()), a.grad.numpy().copy()
        return float(L.detach())

    _, g = loss(a0, grad=True)
    h = 1e-4
    for b in np.argsort(-np.abs(g))[:6]:
        e = np.zeros(nb)
        e[b] = h
        fd = (loss(a0 + e) - loss(a0 - e)) / (2 * h)
        assert abs(fd - g[b]) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(g))), (b, fd, g[b])
    # the data gradient: L is quadratic in d, so central differences along a
    # direction are exact up to rounding and the solver tolerance
    dd = d.clone().requires_grad_(True)
    x = cg.FillRealize.apply(dd, torch.from_numpy(a0), plan, model, [5], 1e-13)
    (x[0] * x[0] * m).sum().backward()
    v = torch.from_numpy(np.random.default_rng(2).standard_normal((n, n))).cuda()

    def loss_d(dv):
        x = cg.FillRealize.apply(dv, torch.from_numpy(a0), plan, model, [5], 1e-13)
        return float((x[0] * x[0] * m).sum())

    fd = (loss_d(d + v) - loss_d(d - v)) / 2.0
    an = float((dd.grad * v).sum())
    assert abs(fd - an) <= 1e-7 * abs(fd)


def test_autograd_backward_after_other_work_reruns_its_forward():
    """Two forwards on one plan, then the first one's backward: the backward
    re-runs its own forward first (the plan's state belongs to the second),
    so its gradient equals a clean single forward/backward."""
    n, nb = 64, 8
    model, plan, obs = _autograd_setup(n, "fp64", nbands=nb)
    d = torch.from_numpy(O.draw(O.hermitian_full(model(np.ones(nb)), n), 6)).cuda()
    m = torch.from_numpy(obs == 0).cuda()
    a1 = torch.ones(nb, dtype=torch.float64, requires_grad=True)
    a2 = torch.full((nb,), 1.2, dtype=torch.float64, requires_grad=True)
    x1 = cg.FillRealize.apply(d, a1, plan, model, [3], 1e-12)
    x2 = cg.FillRealize.apply(d, a2, plan, model, [4], 1e-12)
    (x1[0] * x1[0] * m).sum().backward()
    (x2[0] * x2[0] * m).sum().backward()
    for a, s, ref_a in ((a1, 3, np.ones(nb)), (a2, 4, np.full(nb, 1.2))):
        q, qp, _ = _autograd_setup(n, "fp64", nbands=nb)
        aa = torch.from_numpy(ref_a).requires_grad_(True)
        x = cg.FillRealize.apply(d, aa, qp, q, [s], 1e-12)
        (x[0] * x[0] * m).sum().backward()
        assert torch.equal(a.grad, aa.grad)


# ------------------------------------------------------------------ lanes

@pytest.mark.parametrize("ny,nx", [(128, 128), (60, 140)])
@pytest.mark.parametrize("host_loops", [False, True])
@pytest.mark.parametrize("mode", ["fp32", "fp64", "mixed"])
def test_lanes_do_not_change_results(mode, host_loops, ny, nx):
    """The CG loops' lanes (sub-batches run as parallel branches of the loop
    graph, an update IF node per lane in mixed mode) leave every realization
    and its iteration count bit for bit unchanged: 1, 2 and 3 lanes over a
    batch of 5 (lanes of 3 + 2 and 2 + 2 + 1 instances), on a power-of-two
    and a mixed-radix grid."""
    P = synth.spectrum_cmb_like(ny, nx, 2 * math.pi / max(ny, nx))
    obs = synth.mask_area_target(ny, nx, seed=31) if ny == nx else \
        synth.mask_band_discs(ny, nx, 6, 5, 2.0, 5.0, 31)
    d = torch.from_numpy(O.draw(O.hermitian_full(P, nx), 4)).to(DT[mode]).cuda()
    tol = 1e-6 if mode == "fp32" else 1e-10
    res = []
    for lanes in (1, 2, 3):
        plan = cg.Plan(P, obs, mode=mode, batch=5, lanes=lanes, host_loops=host_loops)
        x, st = plan.realize(d, [10, 11, 12, 13, 14], tol)
        assert all(s["status"] == 0 for s in st)
        res.append((x, [s["iters"] for s in st]))
    for x, it in res[1:]:
        assert torch.equal(x, res[0][0]) and it == res[0][1]


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_lanes_do_not_change_the_adjoint(mode):
    """fill_backward's adjoint solve runs on the same lanes: dL/dd and the
    band gradients are bit for bit those of a one-lane plan."""
    bidx, sig, noise, obs = band_case(64, nbands=8)
    model = cg.BandPowerSpectrum(bidx, sig, noise)
    d = torch.from_numpy(O.draw(O.hermitian_full(model(np.ones(8)), 64), 6)).cuda()
    m = torch.from_numpy(obs == 0).cuda()
    outs = []
    for lanes in (1, 2):
        plan = cg.Plan(model(np.ones(8)), obs, mode=mode, backward=True, batch=2, lanes=lanes)
        plan.set_bands(bidx, sig)
        x, _ = plan.realize(d, [3, 4], 1e-10)
        gd, gb, _ = plan.backward(d, (2.0 * x * m).contiguous(), 1e-10)
        outs.append((gd, gb))
    assert torch.equal(outs[0][0], outs[1][0])
    assert np.array_equal(np.asarray(outs[0][1]), np.asarray(outs[1][1]))
