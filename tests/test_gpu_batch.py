"""GPU batching: many realizations over masks and grid sizes in one call
(fill_group_*), the mixed-size batch workload, and the autotuner."""
import math
import os

import numpy as np
import pytest

import oracle as O
from workloads import synth, WORKLOADS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1109_0286_gb300 as cg  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def mixed_items(sizes, k_lo_n, seed0=13):
    items = []
    k_lo = 2 * math.pi / k_lo_n
    spectra = {}
    for n, count in sizes:
        spectra[n] = synth.spectrum_cmb_like(n, n, k_lo)
        for j in range(count):
            obs = synth.mask_area_target(n, n, seed=seed0 * 100_000 + n * 1000 + j)
            items.append((n, spectra[n], obs))
    return items


@pytest.mark.parametrize("mode", ["fp64", "fp32", "mixed"])
def test_group_equals_single_plans(mode):
    """A group of mixed-size plans gives every realization the single-plan
    path gives (same schedule, same arithmetic), and matches the oracle; in
    mixed mode (reliable updates per class, an update IF node per class) the
    double-float true residual reaches the tolerance."""
    items = mixed_items([(64, 3), (128, 2), (256, 2)], 256)
    dt = torch.float32 if mode == "fp32" else torch.float64
    plans, ds, dn = [], [], []
    for k, (n, P, obs) in enumerate(items):
        plans.append(cg.Plan(P, obs, mode=mode, batch=2 if k == 1 else 1))
        d = O.draw(O.hermitian_full(P, n), 500 + k)
        dn.append(d)
        ds.append(torch.from_numpy(d).to(dtype=dt, device="cuda"))
    g = cg.Group(plans)
    seeds = list(range(7, 7 + g.size))
    tol = {"fp64": 1e-9, "fp32": 1e-6, "mixed": 1e-10}[mode]
    outs, stats = g.realize(ds, seeds, tol)
    if mode == "mixed":
        assert all(0 <= s["true_rel_resid"] <= tol for s in stats)
    flat = 0
    for k, (p, (n, P, obs)) in enumerate(zip(plans, items)):
        xs, _ = p.realize(ds[k], seeds[flat:flat + p.batch], tol)
        assert torch.equal(outs[k], xs), k
        m = obs == 0
        if k < 3:
            ref = O.realize(P, obs, dn[k], seeds[flat], tol=1e-12)
            x = outs[k][0].cpu().numpy().astype(np.float64)
            assert rel(x[m], ref.x[m]) <= (2e-5 if mode == "fp32" else 1e-8)
        flat += p.batch
    assert all(s["status"] == 0 for s in stats)


@pytest.mark.parametrize("mode", ["fp32", "mixed"])
def test_group_host_loops_equal_graph(mode):
    items = mixed_items([(64, 2), (128, 1)], 128, seed0=17)
    dt = torch.float32 if mode == "fp32" else torch.float64
    tol = 1e-6 if mode == "fp32" else 1e-10
    outs = []
    for host in (False, True):
        plans, ds = [], []
        for k, (n, P, obs) in enumerate(items):
            plans.append(cg.Plan(P, obs, mode=mode, host_loops=host))
            d = O.draw(O.hermitian_full(P, n), 600 + k)
            ds.append(torch.from_numpy(d).to(dtype=dt, device="cuda"))
        g = cg.Group(plans)
        outs.append(g.realize(ds, list(range(3, 3 + g.size)), tol))
    for a, b in zip(outs[0][0], outs[1][0]):
        assert torch.equal(a, b)
    assert [s["iters"] for s in outs[0][1]] == [s["iters"] for s in outs[1][1]]


def test_autotune_keeps_results_close(tmp_path):
    n = 256
    P = synth.spectrum_cmb_like(n, n, 2 * math.pi / n)
    obs = synth.mask_area_target(n, n, seed=4)
    d = torch.from_numpy(O.draw(O.hermitian_full(P, n), 1)).cuda()
    a = cg.Plan(P, obs, mode="fp64", batch=2)
    xa, _ = a.realize(d, [3, 4], 1e-10)
    b = cg.Plan(P, obs, mode="fp64", batch=2)
    cache = str(tmp_path / "tune.txt")
    b.autotune(cache)
    assert os.path.exists(cache) and open(cache).read().strip()
    xb, _ = b.realize(d, [3, 4], 1e-10)
    m = torch.from_numpy(obs == 0).cuda()
    assert rel(xb[:, m].cpu().numpy(), xa[:, m].cpu().numpy()) <= 1e-9
    c = cg.Plan(P, obs, mode="fp64", batch=2)
    c.autotune(cache)                     # served from the cache
    xc, _ = c.realize(d, [3, 4], 1e-10)
    assert torch.equal(xb, xc)


def test_batch_mixed_full_workload():
    """256 realizations (128 x 256^2, 96 x 512^2, 32 x 1024^2), own masks at
    5-25% masked area, shared CMB-like P(k), FP32 operator, tol 1e-6, in one
    group call; sampled instances of every size against the oracle."""
    spec = WORKLOADS["batch_mixed"]
    items = mixed_items(spec["sizes"], spec["k_lo_n"], spec["mask_seed"])
    plans, ds, dn = [], [], {}
    for k, (n, P, obs) in enumerate(items):
        plans.append(cg.Plan(P, obs, mode="fp32"))
        if n not in dn:
            dn[n] = O.draw(O.hermitian_full(P, n), spec["data_seed"])
        ds.append(torch.from_numpy(dn[n]).float().cuda())
    g = cg.Group(plans, autotune=True)
    seeds = [spec["seed0"] + i for i in range(g.size)]
    outs, stats = g.realize(ds, seeds, spec["tol"])
    assert g.size == 256 and all(s["status"] == 0 for s in stats)
    firsts = {}
    for k, (n, _, _) in enumerate(items):
        firsts.setdefault(n, k)
    for n, k in firsts.items():
        _, P, obs = items[k]
        ref = O.realize(P, obs, dn[n], seeds[k], tol=spec["tol"])
        x = outs[k][0].cpu().numpy().astype(np.float64)
        m = obs == 0
        assert np.array_equal(x[~m], dn[n].astype(np.float32)[~m].astype(np.float64))
        assert rel(x[m], ref.x[m]) <= 1e-5, (n, rel(x[m], ref.x[m]))


def test_mixed_group_needs_one_reliable_update_threshold():
    """Mixed-mode groups run the reliable-update loop: plans with restarted
    refinement (update_delta = 0) or with different thresholds are refused,
    and fill_realize_batch runs such lists plan by plan instead."""
    items = mixed_items([(64, 2)], 64, seed0=21)
    (_, P0, obs0), (_, P1, obs1) = items
    a = cg.Plan(P0, obs0, mode="mixed", update_delta=0.0)
    b = cg.Plan(P1, obs1, mode="mixed")
    c = cg.Plan(P1, obs1, mode="mixed", update_delta=1e-3)
    for plans in ([a, b], [b, c]):
        with pytest.raises(cg.FillError):
            cg.Group(plans)
    d = torch.from_numpy(O.draw(O.hermitian_full(P0, 64), 5)).cuda()
    outs, stats = cg.realize_batch([a, b], [d, d], [1, 2], 1e-10)
    xa, _ = a.realize(d, [1], 1e-10)
    assert torch.equal(outs[0], xa) and all(s["status"] == 0 for s in stats)
