"""GPU adjoint gradients (fill_backward) against the FP64 oracle's gradient
and against central finite differences of the GPU forward.

Loss: L = sum over masked pixels of x^2 (so dL/dx = 2 x on M, 0 on U);
parameters: the data map d and 32 log-spaced band amplitudes a_b of
P(k) = sum_b a_b 1[k in b] S(k) + N (at a_b = 1).
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def grad_case(n, scale_of=2048, nbands=32, band_frac=0.15, ndiscs=None, seed=14):
    k_lo = 2 * math.pi / (n if scale_of is None else min(n, scale_of))
    bidx, sig, noise = synth.band_templates_half(n, n, k_lo, nbands)
    P = sig + noise
    nd = ndiscs if ndiscs is not None else max(4, 500 * n * n // (2048 * 2048))
    obs = synth.mask_band_discs(n, n, int(round(band_frac * n)), nd, 2.0, 12.0, seed)
    d = O.draw(O.hermitian_full(P, n), 6)
    return P, obs, d, bidx, sig, noise


def gpu_grad(P, obs, d, bidx, sig, mode, seed, tol, batch=1):
    dt = torch.float32 if mode == "fp32" else torch.float64
    plan = cg.Plan(P, obs, mode=mode, backward=True, batch=batch)
    plan.set_bands(bidx, sig)
    dg = torch.from_numpy(d).to(device="cuda", dtype=dt)
    seeds = [seed + i for i in range(batch)]
    x, _ = plan.realize(dg, seeds, tol)
    m = torch.from_numpy(obs == 0).cuda()
    g = (2.0 * x * m).contiguous()
    gd, gb, st = plan.backward(dg, g, tol)
    return x.cpu().numpy(), gd.cpu().numpy(), gb, st, plan


@pytest.mark.parametrize("mode,tol,bound", [("fp64", 1e-12, 1e-8), ("mixed", 1e-11, 1e-7),
                                             ("fp32", 1e-6, 2e-3)])
def test_backward_matches_oracle(mode, tol, bound):
    n = 128
    P, obs, d, bidx, sig, _ = grad_case(n)
    x, gd, gb, st, _ = gpu_grad(P, obs, d, bidx, sig, mode, 7, tol)
    real = O.realize(P, obs, d, 7, tol=1e-13)
    gd_o, gb_o, _ = O.backward(P, obs, d, 7, real, bidx, sig, tol=1e-13)
    u = obs == 1
    e_d, e_b = rel(gd[0][u], gd_o[u]), rel(gb[0], gb_o)
    print(f"{mode}: grad_d {e_d:.2e} grad_bands {e_b:.2e} adjoint iters {st[0]['iters']}")
    assert np.all(gd[0][~u] == 0)
    assert e_d <= bound and e_b <= bound


def test_backward_batch_matches_singles():
    n = 64
    P, obs, d, bidx, sig, _ = grad_case(n)
    _, gd4, gb4, _, _ = gpu_grad(P, obs, d, bidx, sig, "fp64", 3, 1e-12, batch=3)
    for i in range(3):
        _, gd1, gb1, _, _ = gpu_grad(P, obs, d, bidx, sig, "fp64", 3 + i, 1e-12)
        assert rel(gd4[i], gd1[0]) <= 1e-12 and rel(gb4[i], gb1[0]) <= 1e-12


def test_band_gradient_finite_differences():
    """Central differences (step 1e-4) of the GPU FP64 forward at tol 1e-13."""
    n = 64
    P, obs, d, bidx, sig, noise = grad_case(n, nbands=32)
    _, gd, gb, _, _ = gpu_grad(P, obs, d, bidx, sig, "fp64", 5, 1e-13)
    dg = torch.from_numpy(d).cuda()
    m = obs == 0

    def loss(amps):
        plan = cg.Plan(amps[bidx] * sig + noise, obs, mode="fp64")
        x, _ = plan.realize(dg, [5], 1e-13)
        return float(np.sum(x[0].cpu().numpy()[m] ** 2))

    h = 1e-4
    ones = np.ones(32)
    active = [b for b in range(32) if abs(gb[0][b]) > 1e-6 * np.max(np.abs(gb[0]))]
    for b in active[::4]:
        e = np.zeros(32)
        e[b] = h
        fd = (loss(ones + e) - loss(ones - e)) / (2 * h)
        assert abs(fd - gb[0][b]) <= 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(gb[0]))), (b, fd, gb[0][b])


def test_grad2048_full_size():
    """The 2048^2 differentiation workload (FP32 operator, FP64-accurate
    reductions, tol 1e-6) at full size: dL/dd against directional central
    differences (L is quadratic in d, so they have no truncation error) and
    dL/da_b against central differences with step 1e-4, both evaluated with
    the mixed-precision forward refined to 1e-11."""
    P, obs, spec = workload("grad2048")
    n = obs.shape[0]
    bidx, sig, noise = synth.band_templates_half(n, n, spec["k_lo"], spec["nbands"])
    d = O.draw(O.hermitian_full(P, n), spec["data_seed"])
    seed, tol = spec["seeds"][0], spec["tol"]
    x, gd, gb, st, plan = gpu_grad(P, obs, d, bidx, sig, "fp32", seed, tol)
    assert st[0]["status"] == 0
    dg = torch.from_numpy(d).float().cuda()
    m = obs == 0
    mixed = cg.Plan(P, obs, mode="mixed")
    dd = torch.from_numpy(d).cuda()

    def loss(dd_):
        xx, _ = mixed.realize(dd_, [seed], 1e-11)
        return float(np.sum(xx[0].cpu().numpy()[m] ** 2))

    rng = np.random.default_rng(1)
    for _ in range(2):
        v = torch.from_numpy(rng.standard_normal((n, n))).cuda()
        fd = (loss(dd + v) - loss(dd - v)) / 2.0
        an = float(np.sum(gd[0] * v.cpu().numpy()))
        assert abs(fd - an) <= 2e-3 * abs(fd), (fd, an)

    def loss_a(amps):
        pl = cg.Plan(amps[bidx] * sig + noise, obs, mode="mixed")
        xx, _ = pl.realize(dd, [seed], 1e-11)
        pl.close()
        return float(np.sum(xx[0].cpu().numpy()[m] ** 2))

    h = 1e-4
    ones = np.ones(spec["nbands"])
    big = np.argsort(-np.abs(gb[0]))[:3]
    for b in big:
        e = np.zeros(spec["nbands"])
        e[b] = h
        fd = (loss_a(ones + e) - loss_a(ones - e)) / (2 * h)
        assert abs(fd - gb[0][b]) <= 2e-3 * abs(fd), (b, fd, gb[0][b])
    del dg
