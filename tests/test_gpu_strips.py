"""GPU: subdivision of the mask (Sect. 6.2) and noise-boosted strip refinement
(Sect. 6.4) against the oracle."""
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
from paper_1109_0286_gb300 import laplace, strips  # noqa: E402


@pytest.mark.parametrize("name,deltas", [("patch1024", (3.0, 7.0, 15.0, 35.0, 100.0)),
                                         ("wide4096_16", (2.0, 5.0, 9.0, 24.0))])
def test_subdivide_is_bit_exact(name, deltas):
    if name == "wide4096_16":
        _, obs, _ = workload("wide4096", scale=16)
    else:
        _, obs, _ = workload(name)
    dev = torch.from_numpy(np.ascontiguousarray(obs)).cuda()
    for delta in deltas:
        for thr in (0.03, 0.1):
            got = cg.fill_subdivide(dev, delta, thr).cpu().numpy().astype(bool)
            assert np.array_equal(got, O.subdivide(obs, delta, thr)), (delta, thr)


def test_subdivide_rejects_discs_larger_than_the_grid():
    dev = torch.ones((32, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(cg.FillError):
        cg.fill_subdivide(dev, 66.0)


def _strip_case(n=128):
    _, obs, _ = workload("wide4096", scale=4096 // n)
    S = synth.spectrum_lorentz_beam(n, n, k0=2 * math.pi / 16, sb=1.0, noise_frac=0.0)
    N = np.full_like(S, 1e-4 * S.max())
    d = O.draw(O.hermitian_full(S + N, n), 6)
    return S, N, obs, d


@pytest.mark.parametrize("mode,bound", [("fp64", 1e-8), ("mixed", 1e-7)])
def test_strip_refine_matches_oracle(mode, bound):
    S, N, obs, d = _strip_case(128)
    stages = [(2000.0, 24.0), (40.0, 10.0), (1.0, 4.0)]
    x, log = strips.strip_refine(S, N, obs, torch.from_numpy(d).cuda(), stages, mode=mode,
                                 tol=1e-11)
    ref = O.strip_refine(S, N, obs, d, stages, tol=1e-11)
    x = x.cpu().numpy()
    m = obs == 0
    assert np.array_equal(x[~m], d[~m])
    assert np.linalg.norm(x[m] - ref[m]) <= bound * np.linalg.norm(ref[m])
    for (beta, w, npx, iters), (b2, w2) in zip(log, stages):
        assert (beta, w) == (b2, w2) and npx == int(O.subdivide(obs, w).sum()) and iters > 0


# ------------------------------------------------------------------ Laplace interpolation (Sect. 6.1)


def _oracle_laplace(obs_inner, x, tol=1e-12):
    ny, nx = x.shape
    Pl = O.hermitian_full(laplace.stencil_spectrum(ny, nx), nx)
    m = obs_inner == 0
    b = O.rhs(Pl, obs_inner, x, np.zeros_like(x))
    res = O.pcg(lambda v: O.apply_A(v, Pl, m), b,
                lambda v: O.apply_S(O.apply_S(v, Pl, m), Pl, m), tol=tol, max_iter=20000)
    return np.where(m, res.u, x)


@pytest.mark.parametrize("mode,bound", [("fp64", 1e-8), ("mixed", 1e-8)])
def test_laplace_fill_matches_oracle_and_stencil(mode, bound):
    """Harmonic interpolation into a band (the 5-point-stencil ML fill):
    against the oracle, and the stencil equation holds on the band."""
    n = 256
    x = O.draw(O.hermitian_full(synth.spectrum_cmb_like(n, n, 2 * math.pi / n), n), 2)
    inner = laplace.band_rows(n, n, 60)
    got, st = laplace.laplace_fill(inner, torch.from_numpy(x).cuda(), mode=mode, tol=1e-12)
    got = got.cpu().numpy()
    ref = _oracle_laplace(inner, x)
    m = inner == 0
    assert np.array_equal(got[~m], x[~m])
    assert np.linalg.norm(got[m] - ref[m]) <= bound * np.linalg.norm(ref[m])
    lap = 4 * got - (np.roll(got, 1, 0) + np.roll(got, -1, 0) + np.roll(got, 1, 1) +
                     np.roll(got, -1, 1))
    assert np.abs(lap[m]).max() <= 1e-6 * np.abs(got).max()


def test_far_interior_laplace_vs_exact_1024():
    """Sect. 6.1 at 1024^2: a 410-row band (40%) with 82-row boundary layers
    removed; the Laplace interpolation from the exact ML values there differs
    from the ML fill inside by about 5% (L2), the same figure the oracle
    gets, and the paper's "< 5%" scale."""
    n = 1024
    P = synth.spectrum_cmb_like(n, n, 2 * math.pi / 4096)
    d = O.draw(O.hermitian_full(P, n), 3)
    lap, ml, inner, _ = laplace.far_interior(P, torch.from_numpy(d).cuda(), 410, 82,
                                             mode="mixed", tol=1e-8)
    lap, ml = lap.cpu().numpy(), ml.cpu().numpy()
    m = inner == 0
    gpu = np.linalg.norm(lap[m] - ml[m]) / np.linalg.norm(ml[m])
    Pf = O.hermitian_full(P, n)
    outer = laplace.band_rows(n, n, 410)
    mo = outer == 0
    b = O.rhs(Pf, outer, d, np.zeros_like(d))
    res = O.pcg(lambda v: O.apply_A(v, Pf, mo), b,
                lambda v: O.apply_S(O.apply_S(v, Pf, mo), Pf, mo), tol=1e-8)
    ml_o = np.where(mo, res.u, d)
    lap_o = _oracle_laplace(inner, ml_o, tol=1e-10)
    orc = np.linalg.norm(lap_o[m] - ml_o[m]) / np.linalg.norm(ml_o[m])
    assert abs(gpu - orc) <= 2e-3 * orc, (gpu, orc)
    assert gpu < 0.06, gpu


def _ms_case(n=256):
    _, obs, _ = workload("wide4096", scale=4096 // n)
    obs = np.array(obs, dtype=np.uint8)
    yy, xx = np.mgrid[:n, :n]
    obs[(yy - n // 3) ** 2 + (xx - n // 2) ** 2 < (n // 5) ** 2] = 0   # one wide hole
    S = synth.spectrum_lorentz_beam(n, n, k0=2 * math.pi / 24, sb=1.0, noise_frac=0.0)
    d = O.draw(O.hermitian_full(S, n), 11)
    return obs, d


def test_ms_classes_match_oracle():
    obs, _ = _ms_case()
    radii = O.ms_radii()
    got = laplace.ms_classes(torch.from_numpy(obs).cuda(), radii).cpu().numpy()
    ref = O.ms_classes(obs, radii)
    assert np.array_equal(got[obs == 0], ref[obs == 0])
    assert len(np.unique(ref[obs == 0])) >= 5   # several annuli take part


@pytest.mark.parametrize("mode,bound", [("fp64", 1e-11), ("mixed", 1e-10), ("fp32", 2e-5)])
def test_laplace_ms_matches_oracle(mode, bound):
    obs, d = _ms_case()
    radii = O.ms_radii()
    for iters in (0, 1, 12):
        x, st = laplace.laplace_ms(obs, torch.from_numpy(d).cuda(), iters, radii, mode=mode)
        x = x.cpu().numpy()
        ref = O.laplace_ms(obs, d, radii, iters)
        m = obs == 0
        assert np.array_equal(x[~m], d.astype(x.dtype)[~m])
        if iters == 0:
            assert not x[m].any()
            continue
        assert np.linalg.norm(x[m] - ref[m]) <= bound * np.linalg.norm(ref[m]), iters
        assert st["iters"] == iters and st["rel_resid"] >= 0


def test_laplace_ms_constant_map_converges_to_the_constant():
    """Averages of a constant are that constant: the sweeps from 0 rise
    monotonically towards it and stay below it."""
    obs, _ = _ms_case(128)
    radii = O.ms_radii(nk=7)
    d = torch.full((128, 128), 3.0, dtype=torch.float64, device="cuda")
    prev = np.zeros(int((obs == 0).sum()))
    for iters in (5, 20, 80):
        x, _ = laplace.laplace_ms(obs, d, iters, radii, mode="fp64")
        v = x.cpu().numpy()[obs == 0]
        assert np.all(v <= 3.0 + 1e-12) and np.all(v >= prev - 1e-12)
        prev = v
    assert np.max(np.abs(prev - 3.0)) < 3e-2   # within 1% after 80 sweeps


def test_set_annuli_rejects_bad_radii():
    obs, _ = _ms_case(64)
    plan = cg.Plan(np.ones((64, 33)), obs, mode="fp64")
    try:
        for r_in, r_out in (([0.0], [32.0]), ([2.0], [1.5]), ([0.5], [0.9])):
            with pytest.raises(cg.FillError):
                plan.set_annuli(r_in, r_out)
        with pytest.raises(cg.FillError):   # no annuli set yet
            plan.laplace_ms(torch.zeros((64, 64), dtype=torch.float64, device="cuda"), 1,
                            torch.zeros((64, 64), dtype=torch.uint8, device="cuda"))
    finally:
        plan.close()
