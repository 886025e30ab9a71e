"""fill_apply_static: the operator application for callers that cannot
allocate device memory (code inside a memory pool or arena it does not own,
or under an allocator that refuses new allocations).  It must give what the
plan-based fill_apply gives, on consecutive calls that reuse its static
scratch, whether it runs first in a fresh process or after other tests.
"""
import math

import numpy as np
import pytest

import oracle as O
from workloads import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1109_0286_gb300 as cg  # noqa: E402


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("ny,nx", [(256, 256), (64, 128)])
def test_static_apply_matches_plan(ny, nx):
    P = synth.spectrum_cmb_like(ny, nx, 2 * math.pi / max(ny, nx))
    obs = synth.mask_band_discs(ny, nx, ny // 8, 5, 2.0, 6.0, seed=ny + nx)
    plan = cg.Plan(P, obs, mode="fp32")
    P_dev = torch.from_numpy(P).cuda()
    obs_dev = torch.from_numpy(obs).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    Pf = O.hermitian_full(P, nx)
    masked = obs == 0
    rng = np.random.default_rng(ny)
    for call in range(2):                       # two calls in a row reuse the scratch
        xn = rng.standard_normal((ny, nx)).astype(np.float32)
        x = torch.from_numpy(xn).cuda()
        xd = xn.astype(np.float64)
        oracle = [O.apply_power(xd, Pf, -1.0), O.apply_power(xd, Pf, 0.5),
                  O.apply_A(xd, Pf, masked), O.apply_S(xd, Pf, masked)]
        for which in range(4):
            out = torch.empty_like(x)
            cg.fill_apply_static(ny, nx, P_dev.data_ptr(), obs_dev.data_ptr(), which,
                                 x.data_ptr(), out.data_ptr(), stream)
            torch.cuda.synchronize()
            ref = plan.apply(which, x)
            assert rel(out, ref) <= 2e-6, (call, which, rel(out, ref))
            got = out.cpu().numpy().astype(np.float64)
            err = np.linalg.norm(got - oracle[which]) / np.linalg.norm(oracle[which])
            assert err <= 2e-6, (call, which, err)


def test_static_apply_rejects_oversize():
    ny = nx = 2048
    P = torch.ones((ny, nx // 2 + 1), dtype=torch.float64, device="cuda")
    x = torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
    out = torch.empty_like(x)
    with pytest.raises(cg.FillError) as e:
        cg.fill_apply_static(ny, nx, P.data_ptr(), 0, 0, x.data_ptr(), out.data_ptr())
    assert e.value.status == 1 and "too large" in str(e.value)
