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
from paper_1109_0286_gb300 import strips  # noqa: E402


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
