"""GPU: mixed-radix grids (nx/2 and ny products of 2, 3, 5, 7) against the
FP64 oracle, whose transforms are numpy's for any length.

Sizes cover every radix in both transforms, odd ny, a power-of-two row with
a mixed-radix column, the longest transforms (4096 = 8^4 points, in rows and
in columns), and the 7000 x 600 flat-sky workload of Sect. 3 (its
scaled-down versions element by element, the full size by the certificate).
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
from paper_1109_0286_gb300 import laplace  # noqa: E402

SIZES = [(60, 84), (45, 70), (27, 32), (48, 64), (600, 350), (8, 4200), (49, 16),
         (24, 8192), (4096, 24)]   # the last two: 4096-point rows, 4096-point columns


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case(ny, nx, seed=0):
    P = synth.spectrum_cmb_like(ny, nx, 2 * math.pi / max(ny, nx))
    obs = synth.mask_band_discs(ny, nx, max(1, int(round(0.15 * ny))), 4, 1.5, 4.0, seed)
    return P, obs


def gpu_map(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype=dtype, device="cuda")


@pytest.mark.parametrize("ny,nx", SIZES)
@pytest.mark.parametrize("mode,bound", [("fp64", 1e-12), ("mixed", 1e-11), ("fp32", 2e-6)])
def test_draw_matches_oracle(ny, nx, mode, bound):
    P, obs = case(ny, nx)
    plan = cg.Plan(P, obs, mode=mode, batch=2)
    y = plan.draw([5, 2**40 + 7]).cpu().numpy()
    Pf = O.hermitian_full(P, nx)
    for i, s in enumerate([5, 2**40 + 7]):
        assert rel(y[i], O.draw(Pf, s)) <= bound


@pytest.mark.parametrize("ny,nx", SIZES)
@pytest.mark.parametrize("mode,bound", [("fp64", 1e-12), ("mixed", 1e-11), ("fp32", 2e-6)])
def test_operators_match_oracle(ny, nx, mode, bound):
    P, obs = case(ny, nx, seed=ny + nx)
    Pf = O.hermitian_full(P, nx)
    masked = obs == 0
    plan = cg.Plan(P, obs, mode=mode)
    dt = torch.float32 if mode == "fp32" else torch.float64
    x = np.random.default_rng(ny * nx).standard_normal((ny, nx))
    refs = [O.apply_power(x, Pf, -1.0), O.apply_power(x, Pf, 0.5),
            O.apply_A(x, Pf, masked), O.apply_S(x, Pf, masked)]
    for which, ref in enumerate(refs):
        got = plan.apply(which, gpu_map(x, dt)).cpu().numpy()
        assert rel(got, ref) <= bound, (which, rel(got, ref))


@pytest.mark.parametrize("scale", [10, 5])
@pytest.mark.parametrize("mode,bound", [("fp64", 1e-9), ("mixed", 1e-8), ("fp32", 1e-4)])
def test_act_workload_matches_oracle(scale, mode, bound):
    """The Sect. 3 workload at 60 x 700 and 120 x 1400, converged, element by
    element; observed pixels equal the data bit for bit."""
    P, obs, spec = workload("act7000x600", scale=scale)
    ny, nx = obs.shape
    d = O.draw(O.hermitian_full(P, nx), spec["data_seed"])
    tol = 1e-6 if mode == "fp32" else 1e-10
    dt = torch.float32 if mode == "fp32" else torch.float64
    npdt = np.float32 if mode == "fp32" else np.float64
    plan = cg.Plan(P, obs, mode=mode, batch=2)
    out, st = plan.realize(gpu_map(d, dt), spec["seeds"][:2], tol)
    m = obs == 0
    for i, seed in enumerate(spec["seeds"][:2]):
        ref = O.realize(P, obs, d, seed, tol=1e-12)
        x = out[i].cpu().numpy().astype(np.float64)
        assert st[i]["status"] == 0
        assert np.array_equal(x[~m], d.astype(npdt)[~m].astype(np.float64))
        assert rel(x[m], ref.x[m]) <= bound, rel(x[m], ref.x[m])


def test_act_full_size_certificate():
    """7000 x 600, batch 4, mixed refinement to 1e-10 (the benchmark's
    configuration): observed pixels equal the data; the draw equals the
    oracle's; the ML certificate (C^-1 w)_M = 0 holds to ~tol by the
    oracle's operator."""
    P, obs, spec = workload("act7000x600")
    ny, nx = obs.shape
    Pf = O.hermitian_full(P, nx)
    d = O.draw(Pf, spec["data_seed"])
    seeds = spec["seeds"]
    plan = cg.Plan(P, obs, mode="mixed", batch=len(seeds))
    out, stats = plan.realize(gpu_map(d, torch.float64), seeds, spec["tol"])
    m = obs == 0
    for i in (0, len(seeds) - 1):
        x = out[i].cpu().numpy()
        assert np.array_equal(x[~m], d[~m])
        y = O.draw(Pf, seeds[i])
        w = np.where(m, x - y, d - y)
        b = O.rhs(Pf, obs, d, y)
        cert = np.linalg.norm(np.where(m, O.apply_power(w, Pf, -1.0), 0)) / np.linalg.norm(b)
        assert cert <= 3e-10, cert
        assert stats[i]["true_rel_resid"] <= spec["tol"]


@pytest.mark.parametrize("mode,bound", [("fp64", 1e-11), ("mixed", 1e-10), ("fp32", 1e-5)])
def test_relax_and_ml_match_oracle(mode, bound):
    P, obs = case(60, 84, seed=5)
    Pf = O.hermitian_full(P, 84)
    d = O.draw(Pf, 41)
    dt = torch.float32 if mode == "fp32" else torch.float64
    plan = cg.Plan(P, obs, mode=mode)
    m = obs == 0
    out, _ = plan.relax(gpu_map(d, dt), 30)
    ref, _ = O.relax(P, obs, d, 30)
    assert rel(out[0].cpu().numpy().astype(np.float64)[m], ref[m]) <= bound
    tol = 1e-6 if mode == "fp32" else 1e-11
    ml, _ = plan.ml(gpu_map(d, dt), tol)
    dense = O.ml_dense_prec(Pf, obs, d.ravel()[obs.ravel() == 1])
    got = ml[0].cpu().numpy().astype(np.float64).ravel()[m.ravel()]
    assert rel(got, dense) <= (1e-4 if mode == "fp32" else 1e-8)


def test_laplace_ms_matches_oracle():
    obs = synth.mask_band_discs(90, 140, 30, 3, 3.0, 6.0, 2)
    d = O.draw(O.hermitian_full(synth.spectrum_cmb_like(90, 140, 2 * math.pi / 140), 140), 3)
    radii = O.ms_radii(nk=5)
    x, _ = laplace.laplace_ms(obs, torch.from_numpy(d).cuda(), 10, radii, mode="fp64")
    ref = O.laplace_ms(obs, d, radii, 10)
    m = obs == 0
    assert rel(x.cpu().numpy()[m], ref[m]) <= 1e-11


def test_backward_matches_oracle():
    ny, nx = 60, 84
    bidx, sig, noise = synth.band_templates_half(ny, nx, 2 * math.pi / 84, 8)
    P = sig + noise
    obs = synth.mask_band_discs(ny, nx, 9, 3, 2.0, 4.0, 14)
    d = O.draw(O.hermitian_full(P, nx), 6)
    plan = cg.Plan(P, obs, mode="fp64", backward=True)
    plan.set_bands(bidx, sig)
    dg = gpu_map(d, torch.float64)
    x, _ = plan.realize(dg, [7], 1e-12)
    mm = torch.from_numpy(obs == 0).cuda()
    gd, gb, _ = plan.backward(dg, (2.0 * x * mm).contiguous(), 1e-12)
    real = O.realize(P, obs, d, 7, tol=1e-13)
    gd_o, gb_o, _ = O.backward(P, obs, d, 7, real, bidx, sig, tol=1e-13)
    u = obs == 1
    assert rel(gd.cpu().numpy()[0][u], gd_o[u]) <= 1e-8
    assert rel(gb[0], gb_o) <= 1e-8


def test_mixed_radix_sizes_rejected_where_unsupported():
    P, obs = case(60, 84)
    for ny, nx in ((66, 84), (60, 86), (60, 85), (8200, 84), (60, 8400), (6, 84)):
        Pb = synth.spectrum_cmb_like(ny, nx, 0.1)
        ob = np.ones((ny, nx), np.uint8)
        with pytest.raises((cg.FillError, ValueError)):
            cg.Plan(Pb, ob, mode="fp64")
    # groups take mixed-radix plans (tests/test_gpu_boundary.py checks their
    # results), also after the autotuner has changed the plan's schedule
    plan = cg.Plan(P, obs, mode="fp32")
    plan.autotune()
    g = cg.Group([plan])
    assert g.size == 1


@pytest.mark.parametrize("mode,bound", [("fp64", 1e-9), ("mixed", 1e-8)])
def test_every_radix_schedule_matches_oracle(tmp_path, mode, bound):
    """Every radix schedule the autotuner can choose (radix-8 stages or not;
    odd radices ascending or descending), forced through a cache line, gives
    the oracle's converged realization; the autotuner's own choice is written
    to its cache and, served again from there, reproduces itself bit for bit.
    120 x 840: nx/2 = 420 = 4 3 5 7, ny = 120 = 8 3 5."""
    ny, nx = 120, 840
    P, obs = case(ny, nx)
    d = O.draw(O.hermitian_full(P, nx), 9)
    ref = O.realize(P, obs, d, 5, tol=1e-12)
    m = obs == 0
    prec, v = (1, 1) if mode == "fp64" else (0, 2)
    dd = gpu_map(d, torch.float64)
    for rcode in range(4):
        for ccode in range(4):
            cache = tmp_path / f"forced_{mode}_{rcode}{ccode}.txt"
            cache.write_text(f"g {prec} {ny} {nx} 1 {v} {v} {rcode} {ccode}\n")
            plan = cg.Plan(P, obs, mode=mode)
            plan.autotune(str(cache))
            out, st = plan.realize(dd, [5], 1e-10)
            x = out[0].cpu().numpy()
            assert st[0]["status"] == 0
            assert np.array_equal(x[~m], d[~m])
            assert rel(x[m], ref.x[m]) <= bound, (rcode, ccode, rel(x[m], ref.x[m]))
    cache = str(tmp_path / f"tuned_{mode}.txt")
    a = cg.Plan(P, obs, mode=mode)
    a.autotune(cache)
    assert any(line.startswith("g ") for line in open(cache))
    xa, _ = a.realize(dd, [5], 1e-10)
    assert rel(xa[0].cpu().numpy()[m], ref.x[m]) <= bound
    b = cg.Plan(P, obs, mode=mode)
    b.autotune(cache)   # served from the cache
    xb, _ = b.realize(dd, [5], 1e-10)
    assert torch.equal(xa, xb)


def test_schedule_options_set_the_loop_precision():
    """rows_per_cta / ffts_per_cta set the CTA shapes of the CG loop's
    precision; the double-float passes of the mixed mode keep their own
    defaults (on the 7000 x 600 grid their 256-thread groups could not take
    two rows per CTA).  The realization converges like the default plan's."""
    P, obs, spec = workload("act7000x600")
    ny, nx = obs.shape
    d = gpu_map(O.draw(O.hermitian_full(P, nx), spec["data_seed"]), torch.float64)
    outs = []
    for opts in ({}, {"rows_per_cta": 2, "ffts_per_cta": 4}):
        plan = cg.Plan(P, obs, mode="mixed", **opts)
        x, st = plan.realize(d, [spec["seeds"][0]], 1e-10)
        assert st[0]["status"] == 0 and st[0]["true_rel_resid"] <= 1e-10
        outs.append(x[0].cpu().numpy())
    m = obs == 0
    assert rel(outs[1][m], outs[0][m]) <= 1e-8
