#!/usr/bin/env python
"""Benchmark: constrained Gaussian realizations per second (and CG iterations
per second) on the 4096^2 wide-cut workload -- 20% band plus 2000 discs of
radius 2-20 px, a CMB-like P(k), batches of 8 realizations of one data map,
mixed precision (FP32 FFT operator and PCG; draw, right-hand side and true
residuals in double-float arithmetic, about 48 significant bits)
down to a relative residual of 1e-10 -- next to the plain FP64 GPU PCG on the
same inputs and the FP64 CPU oracle on the host cores.

One step = one fill_realize call on a batch of 8 realizations.  Synthetic
inputs: the spectrum and mask recipes of ``workloads`` and a data map drawn
from P(k) on the GPU.  Every timed step streams ~1.5 GB per CG iteration
through HBM, far more than the 129 MB L2, so no L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU runs (torchrun) are replicas: each rank runs its own batches with
its own seeds (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "constrained realizations/s at 4096^2 (rel err <= 1e-5; refined to 1e-10)"
UNIT = "realizations/s"
# FP64 PCG iterations per realization of this workload at tol 1e-10, as the
# FP64 GPU arm of this bench measures them (352.5 over seeds 100-107).  The
# reference arm has no GPU run to measure them in, so it scales the oracle's
# per-iteration time with this count; the GPU arm's cpu_baseline uses the
# count measured in the same run.
FP64_ITERS_WIDE4096 = 352.5

# DRAM traffic (read + write bytes) of one launch of each hot-loop pass, from
# one ncu capture of 2 instances of the 4096^2 workload (FP32 kernels):
# (per-instance MB, shared MB), the shared part (column table, mask words)
# read once per launch; a launch over B instances is B * per-instance +
# shared.  Reported only while the pass-kernel sources hash to the captured
# version; otherwise traffic is null.
TRAFFIC = {"src_hash": "0ebc24cfb84ca3e1",
           "k_col (column FFT, x 1/(nP), inverse FFT)": (104.71, 33.57),
           "k_row src (r, u update + R2C)": (140.56, 4.19),
           "k_row src (p update + R2C)": (88.42, 4.19),
           "k_row sink (C2R + q = P_x, p^T q)": (85.30, 4.19),
           "k_row mid (C2R, P_x, R2C)": (125.08, 4.19)}
KERNEL_SOURCES = ["cg_types.h", "cg_common.cuh", "cg_async.cuh", "cg_fft.cuh", "cg_kernels.cuh",
                  "cg_launch.cuh"]


def kernel_src_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1109_0286_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="wide4096")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 PCG arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp32", "fp64"],
                    help="precision mode of the timed arm (profiling cases)")
    ap.add_argument("--batch", type=int, default=0, help="realizations per step (0: workload's)")
    ap.add_argument("--tol", type=float, default=0.0, help="CG tolerance (0: workload's)")
    ap.add_argument("--no-strips", action="store_true",
                    help="skip the Sect. 6 measurements (strip refinement, far-interior test)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (plain64, patch1024, batch_mixed, grad2048)")
    ap.add_argument("--update-delta", type=float, default=1e-2,
                    help="mixed mode: FP32 residual drop that triggers a true-residual update")
    ap.add_argument("--host-loops", action="store_true",
                    help="launch the CG loops' kernels from the host instead of one graph "
                         "launch per loop (profilers cannot see kernels in conditional nodes)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.lines, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx or None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seeds(seed0, batch, step, rank):
    """Realization seeds of one step of one replica: disjoint across steps
    (stride 100003 per step) and ranks (stride 10000019 per rank) for any
    batch up to 100003 and fewer than 100 steps per rank."""
    return [seed0 + i + 100_003 * step + 10_000_019 * rank for i in range(batch)]


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: the job's time (replicas, max over ranks)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(batch, steps, world, ms_max):
    """Whole-job realizations/s: every rank's realizations over the slowest
    rank's time."""
    return batch * steps * world / (ms_max / 1e3)


def workload_config(name, grid, batch, tol, mode, masked_fraction, world, **extra):
    npix = int(grid[0]) * int(grid[1])
    cfg = {"workload": name, "grid": list(grid), "batch": batch, "tol": tol, "mode": mode,
           "precond": "sqrtC", "masked_fraction": round(float(masked_fraction), 4),
           "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (no flush)",
           # CG-loop lanes of the library's automatic setting (fill_opts.lanes = 0)
           "lanes": 2 if batch >= 2 and npix >= 1 << 20 else 1}
    cfg.update(extra)
    return cfg


def strips_measurement():
    """Noise-boosted strip refinement (Sect. 6.4) with the paper's four
    (beta, w) stages on the 1024^2 patch workload (10% band of 102 rows,
    discs of radius 2-12: masks no wider than the paper's ~100-pixel limit),
    mixed precision: wall time, CG iterations per stage, and the distance to
    the exact ML fill (fill_ml to 1e-8) over the mask and in the last strip.
    The oracle runs the same procedure on the 256^2 version, timed beside the
    GPU on that size."""
    import numpy as np
    import torch
    import oracle as O
    import paper_1109_0286_gb300 as cg
    from paper_1109_0286_gb300 import strips
    from workloads import synth, workload

    def case(scale):
        P, obs, spec = workload("patch1024", scale=scale)
        N = np.full_like(P, synth.cmb_noise_level(spec["k_lo"]))
        plan = cg.Plan(P, obs, mode="mixed")
        d = plan.draw([spec["data_seed"]])[0].clone()      # data drawn from P(k)
        plan.close()
        return P - N, N, obs, d

    out = {"workload": "patch1024 (1024^2, 10% band + 200 discs)", "stages": strips.PAPER_STAGES,
           "mode": "mixed", "tol": 1e-8}
    S, N, obs, dd = case(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, log = strips.strip_refine(S, N, obs, dd, mode="mixed", tol=1e-8)
    torch.cuda.synchronize()
    out["ms"] = (time.perf_counter() - t0) * 1e3
    out["cg_iters_per_stage"] = [entry[3] for entry in log]
    out["strip_pixels"] = [entry[2] for entry in log]
    plan = cg.Plan(S + N, obs, mode="mixed")
    ml, _ = plan.ml(dd, 1e-8)
    plan.close()
    x, ml = x.cpu().numpy(), ml[0].cpu().numpy()
    m = obs == 0
    last = cg.fill_subdivide(torch.from_numpy(obs).cuda(), strips.PAPER_STAGES[-1][1])
    last = last.cpu().numpy().astype(bool)
    out["rel_err_mask"] = float(np.linalg.norm(x[m] - ml[m]) / np.linalg.norm(ml[m]))
    out["rel_err_last_strip"] = float(np.linalg.norm(x[last] - ml[last]) / np.linalg.norm(ml[last]))
    # CPU baseline leg: the oracle runs the same procedure on the 256^2 version
    S4, N4, obs4, d4 = case(4)
    stages4 = [(b, w / 4.0) for b, w in strips.PAPER_STAGES]
    t0 = time.perf_counter()
    strips.strip_refine(S4, N4, obs4, d4, stages4, mode="mixed", tol=1e-8)
    torch.cuda.synchronize()
    g4 = (time.perf_counter() - t0) * 1e3
    d4h = d4.cpu().numpy()
    t0 = time.perf_counter()
    O.strip_refine(S4, N4, obs4, d4h, stages4, tol=1e-8)
    o4 = (time.perf_counter() - t0) * 1e3
    out["at_256"] = {"gpu_ms": g4, "stages": stages4,
                     "cpu_baseline": {"ms": o4, "cores": threads_used(), "kind": "oracle"}}
    return out


def far_interior_measurement():
    """Sect. 6.1 at 4096^2: the exact ML fill of the 819-row band (20%), then
    the Laplace interpolation into its interior after removing 82 rows along
    each boundary: the relative L2 and max difference inside, and the time."""
    import numpy as np
    import torch
    import paper_1109_0286_gb300 as cg
    from paper_1109_0286_gb300 import laplace
    from workloads import synth
    n, rows, layer = 4096, 819, 82
    P = synth.spectrum_cmb_like(n, n, 2 * np.pi / 4096)
    plan = cg.Plan(P, laplace.band_rows(n, n, rows), mode="mixed")
    dd = plan.draw([3])[0].clone()                          # data drawn from P(k)
    plan.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lap, ml, inner, (sm, sl) = laplace.far_interior(P, dd, rows, layer, mode="mixed", tol=1e-8)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    m = torch.from_numpy(inner == 0).cuda()
    diff = (lap - ml)[m]
    ref = ml[m]
    return {"grid": [n, n], "band_rows": rows, "layer_rows": layer, "mode": "mixed", "ms": ms,
            "ml_iters": sm["iters"], "laplace_iters": sl["iters"],
            "rel_l2": float(torch.linalg.norm(diff) / torch.linalg.norm(ref)),
            "max_rel": float(diff.abs().max() / ref.abs().max())}


def laplace_ms_measurement():
    """The kernel-based Laplace solver of Sect. 6.3 at 4096^2 on the 819-row
    band (20%) with 13 annuli (the largest disc, radius 359, fits the band's
    half-width): ms per sweep (FP32) and the distance to the exact 5-point
    Laplace fill after 50/100/200/400 sweeps, beside the single 3x3 kernel
    (plain Jacobi).  The oracle runs the 512^2 version (102-row band, 8
    annuli) for 50 sweeps, timed beside the GPU."""
    import numpy as np
    import torch
    import oracle as O
    import paper_1109_0286_gb300 as cg
    from paper_1109_0286_gb300 import laplace
    from workloads import synth

    def case(n, rows):
        P = synth.spectrum_cmb_like(n, n, 2 * np.pi / 4096)
        obs = laplace.band_rows(n, n, rows)
        plan = cg.Plan(P, obs, mode="mixed")
        d = plan.draw([3])[0].clone()                       # data drawn from P(k)
        plan.close()
        return obs, d

    def sweeps(plan, d, cls, k):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, _ = plan.laplace_ms(d, k, cls)
        torch.cuda.synchronize()
        return x[0], (time.perf_counter() - t0) * 1e3

    n, rows = 4096, 819
    obs, d = case(n, rows)
    exact, st = laplace.laplace_fill(obs, d, mode="mixed", tol=1e-10)
    m = torch.from_numpy(obs == 0).cuda()
    ref = exact[m]
    out = {"grid": [n, n], "band_rows": rows, "mode": "fp32", "exact_cg_iters": st["iters"]}
    d32 = d.float().contiguous()
    for nk, ks in ((13, (50, 100, 200, 400)), (1, (400,))):
        radii = laplace.ms_radii(nk=nk)
        plan = cg.Plan(np.ones((n, n // 2 + 1)), obs, mode="fp32")
        plan.set_annuli([r[0] for r in radii], [r[1] for r in radii])
        cls = laplace.ms_classes(torch.from_numpy(obs).cuda(), radii)
        sweeps(plan, d32, cls, 2)                            # warm-up
        errs = {}
        for k in ks:
            x, ms = sweeps(plan, d32, cls, k)
            errs[k] = float(torch.linalg.norm(x[m].double() - ref) / torch.linalg.norm(ref))
        plan.close()
        out[f"annuli_{nk}"] = {"rel_l2_vs_exact": errs, "ms_per_sweep": ms / ks[-1],
                               "r_out_max": radii[-1][1]}
    # CPU baseline leg: the oracle on the 512^2 version, 50 sweeps
    obs5, d5 = case(512, 102)
    radii5 = laplace.ms_radii(nk=8)
    d5h = d5.cpu().numpy()
    t0 = time.perf_counter()
    laplace.laplace_ms(obs5, d5, 50, radii5, mode="fp32")
    torch.cuda.synchronize()
    g5 = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    O.laplace_ms(obs5, d5h, radii5, 50)
    o5 = (time.perf_counter() - t0) * 1e3
    out["at_512"] = {"sweeps": 50, "annuli": 8, "gpu_ms_incl_setup": g5,
                     "cpu_baseline": {"ms": o5, "cores": threads_used(), "kind": "oracle"}}
    return out


def act_measurement():
    """The flat-sky season map of Sect. 3 (7000 x 600, ~400 point-source
    holes, a mixed-radix grid), 4 maps per step, mixed precision refined to
    1e-10, with and without the preconditioner (the paper ran plain CG and
    reports 20 minutes per map on one processor, residual halving per
    iteration): realizations/s by CUDA events over 3 steps after 2 warm-up
    steps, iterations per map, the worst true residual, and the oracle timed
    on one host core (draw + right-hand side, one CG iteration, scaled)."""
    import numpy as np
    import torch
    import paper_1109_0286_gb300 as cg
    from workloads import workload
    P, obs, spec = workload("act7000x600")
    ny, nx = obs.shape
    B, tol = len(spec["seeds"]), spec["tol"]
    out = {"grid": [ny, nx], "batch": B, "tol": tol, "mode": "mixed",
           "masked_fraction": float((obs == 0).mean()),
           "paper": "1200 s per map, plain CG, one processor (2011), residual x0.5 per iteration"}
    d = None
    for precond in (True, False):
        plan = cg.Plan(P, obs, mode="mixed", batch=B, precond=precond)
        if d is None:
            d = plan.draw([spec["data_seed"]])[0].clone()   # data drawn from P(k)
        for k in range(2):
            plan.realize(d, [s + 10 * k for s in spec["seeds"]], tol)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters, worst = 0, 0.0
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(3):
            _, st = plan.realize(d, [s + 100 + 10 * k for s in spec["seeds"]], tol)
            iters += sum(x["iters"] for x in st)
            worst = max([worst] + [x["true_rel_resid"] for x in st])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        out["precond" if precond else "plain_cg"] = {
            "realizations_per_s": B / (ms / 1e3), "ms_per_step": ms,
            "iters_per_realization": iters / (3 * B), "worst_true_rel_resid": worst}
        if precond:   # the mixed-radix passes (FP32), CUDA events on the plan's stream
            out["passes"] = {}
            for pid, name in enumerate(("k_col_gen", "k_row_gen src (r, u update + R2C)",
                                        "k_row_gen src (p update + R2C)",
                                        "k_row_gen sink (C2R + q = P_x, p^T q)",
                                        "k_row_gen mid (C2R, P_x, R2C)")):
                pms, pbytes = plan.time_pass(pid, reps=10)
                out["passes"][name] = {"ms": round(pms, 4),
                                       "GB/s": round(pbytes / pms / 1e6, 1)}
        plan.close()
    return out, P, obs, d, spec


def _events_ms(fn, reps):
    """Average device time of fn() over `reps` calls (CUDA events on the
    current stream, after one untimed call)."""
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = [fn() for _ in range(reps)]
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out[-1]


def configs_measurement():
    """The other workloads of the benchmark's configuration list, each timed
    by CUDA events (inputs resident, data drawn from P(k) by the library):

    * plain64: the plain method in FP64 on 64^2, tol 1e-8, one realization;
    * patch1024: 1024^2, FP32 operator with FP64-accurate reductions, tol 1e-6;
    * batch_mixed: 256 realizations (128 x 256^2, 96 x 512^2, 32 x 1024^2),
      each with its own mask, in ONE group call (fill_group_realize, the
      machinery of fill_realize_batch; FP32, tol 1e-6, autotuned size
      classes running as concurrent branches of one graph per CG loop);
      and the same batch in mixed precision to 1e-10 (batch_mixed_refined);
    * grad2048: 2048^2, FP32, 32 band powers: forward, adjoint (fill_backward
      for dL/dd and dL/da_b of L = sum over M of x^2), fill_set_spectrum plus
      forward, and the same through the torch.autograd.Function.
    Returns the dict and the arrays the CPU legs re-check against the oracle."""
    import math
    import numpy as np
    import torch
    import paper_1109_0286_gb300 as cg
    from workloads import synth, workload, WORKLOADS
    out, keep = {}, {}

    for name, reps in (("plain64", 20), ("patch1024", 5)):
        P, obs, spec = workload(name)
        mode = spec["precision"]
        plan = cg.Plan(P, obs, mode=mode)
        d = plan.draw([spec["data_seed"]])[0].clone()
        seed, tol = spec["seeds"][0], spec["tol"]
        ms, (x, st) = _events_ms(lambda: plan.realize(d, [seed], tol), reps)
        out[name] = {"grid": list(obs.shape), "mode": mode, "tol": tol,
                     "realizations_per_s": 1e3 / ms, "ms_per_realization": ms,
                     "iters": st[0]["iters"], "cg_iters_per_s": st[0]["iters"] / (ms / 1e3),
                     "status": st[0]["status"]}
        keep[name] = (P, obs, d.double().cpu().numpy(), x[0].double().cpu().numpy(), seed, tol)
        plan.close()

    spec = WORKLOADS["batch_mixed"]
    k_lo = 2 * math.pi / spec["k_lo_n"]
    plans, ds, sizes = [], [], []
    for n, count in spec["sizes"]:
        P = synth.spectrum_cmb_like(n, n, k_lo)
        first = None
        for j in range(count):
            obs = synth.mask_area_target(n, n, seed=spec["mask_seed"] * 100_000 + n * 1000 + j)
            plans.append(cg.Plan(P, obs, mode="fp32"))
            if first is None:
                first = plans[-1].draw([spec["data_seed"]])[0].clone()
            ds.append(first)
            sizes.append(n)
    g = cg.Group(plans, autotune=True)          # size classes with tuned schedules
    seeds = [spec["seed0"] + i for i in range(len(plans))]
    ms, (_, st) = _events_ms(lambda: g.realize(ds, seeds, spec["tol"]), 2)
    g.close()
    iters = sum(x["iters"] for x in st)
    per_size = {}
    for n in sorted(set(sizes)):
        idx = [i for i, s_ in enumerate(sizes) if s_ == n]
        pl = plans[idx[0]]
        nbytes = sum(pl.time_pass(pid, reps=5)[1] * k for pid, k in ((0, 3), (1, 1), (2, 1), (3, 2), (4, 1)))
        per_size[n] = {"count": len(idx), "iters_mean": sum(st[i]["iters"] for i in idx) / len(idx),
                       "bytes_per_iter": nbytes}
    moved = sum(per_size[sizes[i]]["bytes_per_iter"] * st[i]["iters"] for i in range(len(plans)))
    out["batch_mixed"] = {"realizations": len(plans), "mode": "fp32", "tol": spec["tol"],
                          "realizations_per_s": len(plans) / (ms / 1e3), "ms_per_call": ms,
                          "cg_iters_per_s": iters / (ms / 1e3),
                          "algorithmic_GB_per_s": moved / (ms / 1e3) / 1e9,
                          "all_ok": all(x["status"] == 0 for x in st),
                          "per_size": {str(k): v for k, v in per_size.items()},
                          "note": "one fill_group_realize call; algorithmic bytes = "
                                  "sum of iterations x the per-iteration pass bytes"}
    for p_ in plans:
        p_.close()
    del plans, ds
    torch.cuda.empty_cache()

    # the same 256 realizations in mixed precision (FP32 operator, double-float
    # draw, right-hand side and reliable updates) to 1e-10, one group call
    plans, ds = [], []
    for n, count in spec["sizes"]:
        P = synth.spectrum_cmb_like(n, n, k_lo)
        first = None
        for j in range(count):
            obs = synth.mask_area_target(n, n, seed=spec["mask_seed"] * 100_000 + n * 1000 + j)
            plans.append(cg.Plan(P, obs, mode="mixed"))
            if first is None:
                first = plans[-1].draw([spec["data_seed"]])[0].clone()
            ds.append(first)
    g = cg.Group(plans, autotune=True)
    ms, (_, st) = _events_ms(lambda: g.realize(ds, seeds, 1e-10), 2)
    g.close()
    out["batch_mixed_refined"] = {
        "realizations": len(plans), "mode": "mixed", "tol": 1e-10,
        "realizations_per_s": len(plans) / (ms / 1e3), "ms_per_call": ms,
        "cg_iters_per_s": sum(x["iters"] for x in st) / (ms / 1e3),
        "worst_true_rel_resid": max(x["true_rel_resid"] for x in st),
        "all_ok": all(x["status"] == 0 for x in st),
        "note": "one fill_group_realize call in mixed precision (not the configuration's FP32 "
                "mode): the batching pattern at the precision target of the 4096^2 workload"}
    for p_ in plans:
        p_.close()
    del plans, ds
    torch.cuda.empty_cache()

    P, obs, spec = workload("grad2048")
    n = obs.shape[0]
    bidx, sig, noise = synth.band_templates_half(n, n, spec["k_lo"], spec["nbands"])
    model = cg.BandPowerSpectrum(bidx, sig, noise)
    plan = cg.Plan(P, obs, mode="fp32", backward=True)
    plan.set_bands(bidx, sig)
    d = plan.draw([spec["data_seed"]])[0].clone()
    seed, tol = spec["seeds"][0], spec["tol"]
    m = torch.from_numpy(obs == 0).cuda()
    ms_f, (x, _) = _events_ms(lambda: plan.realize(d, [seed], tol), 3)
    gx = (2.0 * x * m).contiguous()
    ms_b, (_, _, sb) = _events_ms(lambda: plan.backward(d, gx, tol), 3)
    amps = np.linspace(0.9, 1.1, spec["nbands"])

    def respectrum():
        plan.set_spectrum(model(amps))
        return plan.realize(d, [seed], tol)
    ms_s, _ = _events_ms(respectrum, 3)
    a = torch.ones(spec["nbands"], dtype=torch.float64, requires_grad=True)

    def autograd_step():
        xx = cg.FillRealize.apply(d, a, plan, model, [seed], tol)
        (xx[0] * xx[0] * m).sum().backward()
        return xx
    ms_a, _ = _events_ms(autograd_step, 3)
    out["grad2048"] = {"grid": [n, n], "mode": "fp32", "tol": tol, "nbands": spec["nbands"],
                       "forward_ms": ms_f, "backward_ms": ms_b, "adjoint_iters": sb[0]["iters"],
                       "set_spectrum_plus_forward_ms": ms_s,
                       "autograd_forward_backward_ms": ms_a}
    plan.close()
    return out, keep


def cufft_pcg_realize(P_half, masked, d, y, tol, precond=True, max_iter=5000, check_every=8):
    """Timed comparison only, never part of the library: the same constrained
    realization (Sects. 2.1-2.4) written with PyTorch's FFT (cuFFT on the GPU)
    and elementwise ops.  P_half (ny, nx/2+1), masked (ny, nx) bool, d (ny, nx)
    and the draws y (B, ny, nx) are tensors on one device, in one real dtype.
    PCG with B = S S (S = P_x C^{1/2} P_x) until ||r|| <= tol ||b|| for every
    map (tested every `check_every` iterations).  Returns (x, iterations)."""
    import torch
    ny, nx = masked.shape
    m = masked.to(d.dtype)
    Pinv, Psq = 1.0 / P_half, torch.sqrt(P_half)

    def apply(x, Ps):   # C^s x = F^-1 diag(P^s) F x (irfft2 carries 1/n)
        return torch.fft.irfft2(torch.fft.rfft2(x) * Ps, s=(ny, nx))

    def A(v):
        return m * apply(m * v, Pinv)

    def prec(v):
        return m * apply(m * apply(m * v, Psq), Psq) if precond else v

    def dot(a, b):
        return (a * b).sum(dim=(1, 2))

    b = -m * apply((1.0 - m) * (d - y), Pinv)
    u = torch.zeros_like(b)
    r = b.clone()
    z = prec(r)
    p = z.clone()
    rz = dot(r, z)
    thr = tol * tol * dot(b, b)
    it = 0
    while it < max_iter:
        q = A(p)
        pq = dot(p, q)
        alpha = torch.where(pq > 0, rz / pq, torch.zeros_like(pq))[:, None, None]
        u += alpha * p
        r -= alpha * q
        it += 1
        if it % check_every == 0 and bool((dot(r, r) <= thr).all()):
            break
        z = prec(r)
        rz_new = dot(r, z)
        beta = torch.where(rz > 0, rz_new / rz, torch.zeros_like(rz))[:, None, None]
        rz = rz_new
        p = z + beta * p
    return torch.where(masked, y + u, d), it


def cufft_refined_realize(P_half, masked, d, y, tol, inner_tol=1e-5, max_outer=20):
    """Timed comparison only: the same realization with PyTorch FFT (cuFFT)
    in the library's mixed-precision scheme -- FP32 PCG solves of
    A delta = r inside an FP64 iterative refinement (r = b - A u recomputed
    with FP64 transforms) until ||r|| <= tol ||b||.  P_half, d, y: FP64
    tensors; masked: bool.  Returns (x, inner iterations, outer steps)."""
    import torch
    ny, nx = masked.shape
    m64 = masked.to(torch.float64)
    Pinv64 = 1.0 / P_half

    def A64(v):
        return m64 * torch.fft.irfft2(torch.fft.rfft2(m64 * v) * Pinv64, s=(ny, nx))

    b = -m64 * torch.fft.irfft2(torch.fft.rfft2((1.0 - m64) * (d - y)) * Pinv64, s=(ny, nx))
    bn = torch.sqrt((b * b).sum(dim=(1, 2)))
    u = torch.zeros_like(b)
    P32, zeros32 = P_half.float(), torch.zeros_like(b, dtype=torch.float32)
    inner = outer = 0
    for outer in range(1, max_outer + 1):
        r = b - A64(u)
        if bool((torch.sqrt((r * r).sum(dim=(1, 2))) <= tol * bn).all()):
            break
        delta, it = cufft_pcg_solve(P32, masked, r.float(), inner_tol)
        inner += it
        u = u + delta.double()
    return torch.where(masked, y + u, d), inner, outer


def cufft_pcg_solve(P_half, masked, b, tol, precond=True, max_iter=5000, check_every=8):
    """PCG with B = S S on A u = b (PyTorch FFT, the dtype of b) until
    ||r|| <= tol ||b|| for every map.  Returns (u, iterations)."""
    import torch
    ny, nx = masked.shape
    m = masked.to(b.dtype)
    Pinv, Psq = 1.0 / P_half, torch.sqrt(P_half)

    def apply(x, Ps):
        return torch.fft.irfft2(torch.fft.rfft2(x) * Ps, s=(ny, nx))

    def A(v):
        return m * apply(m * v, Pinv)

    def prec(v):
        return m * apply(m * apply(m * v, Psq), Psq) if precond else v

    def dot(a, c):
        return (a * c).sum(dim=(1, 2))

    u = torch.zeros_like(b)
    r = b.clone()
    z = prec(r)
    p = z.clone()
    rz = dot(r, z)
    thr = tol * tol * dot(b, b)
    it = 0
    while it < max_iter:
        q = A(p)
        pq = dot(p, q)
        alpha = torch.where(pq > 0, rz / pq, torch.zeros_like(pq))[:, None, None]
        u += alpha * p
        r -= alpha * q
        it += 1
        if it % check_every == 0 and bool((dot(r, r) <= thr).all()):
            break
        z = prec(r)
        rz_new = dot(r, z)
        beta = torch.where(rz > 0, rz_new / rz, torch.zeros_like(rz))[:, None, None]
        rz = rz_new
        p = z + beta * p
    return u, it


def cufft_arm(P, obs, d, batch, tol64):
    """cuFFT-based PCG timed beside the library (spec comparison):
    FP32 to 1e-5 on `batch` maps, FP64 to tol64 on one map; each timed
    realization includes its draw (torch.randn + one transform pair), the
    right-hand side, the PCG loop and the assembly.  One warm-up realization
    each, then one timed by CUDA events."""
    import torch
    out = {"note": "PyTorch FFT (cuFFT) + elementwise ops; comparison only"}
    try:   # the library's own scheme with cuFFT: FP32 PCG inside FP64 refinement to tol64
        dev = torch.device("cuda")
        Ph = torch.as_tensor(P, dtype=torch.float64, device=dev)
        masked = torch.as_tensor(obs == 0, device=dev)
        dd = d.to(dtype=torch.float64)
        ny, nx = masked.shape

        def refined(seed):
            g = torch.Generator(device=dev).manual_seed(seed)
            xi = torch.randn((batch, ny, nx), generator=g, dtype=torch.float64, device=dev)
            y = torch.fft.irfft2(torch.fft.rfft2(xi) * torch.sqrt(Ph), s=(ny, nx))
            return cufft_refined_realize(Ph, masked, dd, y, tol64)

        refined(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, inner, outer = refined(2)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["fp32_pcg_fp64_refined"] = {"realizations_per_s": batch / (ms / 1e3), "ms_per_step": ms,
                                        "batch": batch, "tol": tol64, "inner_iters": inner,
                                        "refinement_steps": outer, "inner_tol": 1e-5}
    except Exception as e:   # comparison only: never fail the bench line
        out["fp32_pcg_fp64_refined"] = {"error": repr(e)[:200]}
    torch.cuda.empty_cache()
    for name, dt, B, tol in (("fp32", torch.float32, batch, 1e-5), ("fp64", torch.float64, 1, tol64)):
        try:
            dev = torch.device("cuda")
            Ph = torch.as_tensor(P, dtype=dt, device=dev)
            masked = torch.as_tensor(obs == 0, device=dev)
            dd = d.to(dtype=dt)
            ny, nx = masked.shape

            def one(seed):
                g = torch.Generator(device=dev).manual_seed(seed)
                xi = torch.randn((B, ny, nx), generator=g, dtype=dt, device=dev)
                y = torch.fft.irfft2(torch.fft.rfft2(xi) * torch.sqrt(Ph), s=(ny, nx))
                return cufft_pcg_realize(Ph, masked, dd, y, tol, max_iter=2000)

            one(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, it = one(2)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[name] = {"realizations_per_s": B / (ms / 1e3), "ms_per_step": ms, "batch": B,
                         "tol": tol, "iters": it}
        except Exception as e:   # comparison only: never fail the bench line
            out[name] = {"error": repr(e)[:200]}
        torch.cuda.empty_cache()
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def oracle_sample(P, obs, d, seed, iters):
    """Times the FP64 CPU oracle on the full-size workload: the draw and the
    right-hand side once, then `iters` preconditioned CG iterations."""
    import numpy as np
    import oracle as O
    nx = obs.shape[1]
    Pf = O.hermitian_full(P, nx)
    masked = obs == 0
    t0 = time.perf_counter()
    y = O.draw(Pf, seed)
    b = O.rhs(Pf, obs, d, y)
    t1 = time.perf_counter()
    A = lambda v: O.apply_A(v, Pf, masked)                                     # noqa: E731
    B = lambda v: O.apply_S(O.apply_S(v, Pf, masked), Pf, masked)               # noqa: E731
    res = O.pcg(A, b, B, tol=0.0, max_iter=iters)
    t2 = time.perf_counter()
    assert res.iters == iters and np.isfinite(res.u).all()
    return t1 - t0, (t2 - t1) / iters


def threads_used():
    """Host threads the oracle's transforms run on (its own C FFT splits rows
    and columns over every host core; its element-wise NumPy steps run on
    one)."""
    import oracle as O
    return O.threads()


def oracle_check(P, obs, d_np, x_np, seed, tol):
    """The error of one GPU realization against the FP64 oracle on the same
    inputs: the oracle's draw y for the seed, its right-hand side b, and the
    certificate ||b - A u|| / ||b|| of the GPU's correction u = x - y on the
    masked pixels, with the oracle's own operator A (no solve needed at full
    size); also the draw's relative error on M and whether the observed
    pixels equal the data bit for bit."""
    import numpy as np
    import oracle as O
    nx = obs.shape[1]
    Pf = O.hermitian_full(P, nx)
    m = obs == 0
    t0 = time.perf_counter()
    y = O.draw(Pf, seed)
    b = O.rhs(Pf, obs, d_np, y)
    u = np.where(m, x_np - y, 0.0)
    r = b - O.apply_A(u, Pf, m)
    return {"true_rel_resid_oracle": float(np.linalg.norm(r) / np.linalg.norm(b)),
            "observed_bit_exact": bool(np.array_equal(x_np[~m], d_np[~m])),
            "tol": tol, "seed": int(seed), "ms": (time.perf_counter() - t0) * 1e3}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    from workloads import workload
    P, obs, spec = workload(args.workload)
    Pf = O.hermitian_full(P, obs.shape[1])
    d = O.draw(Pf, spec["data_seed"])
    nx = obs.shape[1]
    masked = obs == 0
    t0 = time.perf_counter()
    b = O.rhs(Pf, obs, d, O.draw(Pf, spec["seeds"][0]))
    setup = time.perf_counter() - t0
    A = lambda v: O.apply_A(v, Pf, masked)                                     # noqa: E731
    Bp = lambda v: O.apply_S(O.apply_S(v, Pf, masked), Pf, masked)              # noqa: E731
    per_iter = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.pcg(A, b, Bp, tol=0.0, max_iter=1)
        if k >= args.warmup:
            per_iter.append(time.perf_counter() - t0)
    t_iter = sum(per_iter) / len(per_iter)
    t_real = setup + FP64_ITERS_WIDE4096 * t_iter
    value = 1.0 / t_real
    cores = threads_used()
    sample = (f"FP64 oracle (own C FFT on {cores} host threads, NumPy element-wise steps) "
              f"on {obs.shape[0]}x{obs.shape[1]}: draw + RHS once "
              f"({setup:.1f} s) and 1 preconditioned CG iteration per step "
              f"({t_iter:.1f} s); realizations/s = 1/(setup + {FP64_ITERS_WIDE4096} iterations)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_iter * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {k: v for k, v in workload_config(
                args.workload, obs.shape, args.batch or len(spec["seeds"]), args.tol or spec["tol"],
                "oracle-fp64", masked.mean(), 1,
                sample="one realization's draw and right-hand side, "
                       "iterations timed one per step").items() if k != "lanes"},
            "cg_iters_per_s": 1.0 / t_iter,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import numpy as np
    import torch
    import paper_1109_0286_gb300 as cg
    from workloads import workload

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    P, obs, spec = workload(args.workload)
    ny, nx = obs.shape
    B = args.batch or len(spec["seeds"])
    tol = args.tol or spec["tol"]
    mode = args.mode
    fdt = torch.float32 if mode == "fp32" else torch.float64
    esz = 4 if mode == "fp32" else 8
    plan = cg.Plan(P, obs, mode=mode, batch=B, host_loops=args.host_loops,
                   update_delta=args.update_delta, history_cap=2048)
    d = plan.draw([spec["data_seed"]] * B)[0].clone()       # data drawn from P(k)
    seeds = lambda k: replica_seeds(spec["seeds"][0], B, k, rank)  # noqa: E731

    for k in range(args.warmup):
        plan.realize(d, seeds(k), tol)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, launches, worst_resid = 0, 0, 0.0
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0.record(stream)
        for k in range(args.steps):
            last_x, st = plan.realize(d, seeds(args.warmup + k), tol)
            iters += sum(s["iters"] for s in st)
            launches += st[0]["launches"]
            worst_resid = max([worst_resid] + [s["true_rel_resid"] if s["true_rel_resid"] >= 0
                                               else s["rel_resid"] for s in st])
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    last_seed = seeds(args.warmup + args.steps - 1)[0]
    last_x = last_x[0].clone()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(B, args.steps, world, ms_max)
    iters_per_s = iters * world / (ms_max / 1e3)

    # end to end through the public API with host buffers: every step copies
    # its input map host->device and its realizations device->host (pinned
    # buffers, counted below).  The copies run on a side stream with two
    # buffer sets, so step k's results go back while step k+1 computes, as a
    # serving pipeline would; the timed region ends when the last copy lands.
    d_host = d.cpu().pin_memory()
    out_host = [torch.empty((B, ny, nx), dtype=fdt).pin_memory() for _ in range(2)]
    out_dev = [torch.empty((B, ny, nx), dtype=fdt, device="cuda") for _ in range(2)]
    d_dev = [torch.empty_like(d) for _ in range(2)]
    main, copy = torch.cuda.current_stream(), torch.cuda.Stream()
    h2d = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    d2h = [torch.cuda.Event() for _ in range(2)]
    esteps = max(2, min(args.steps, 4))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(copy):
        d_dev[0].copy_(d_host, non_blocking=True)
        h2d[0].record(copy)
    for k in range(esteps):
        i, j = k % 2, (k + 1) % 2
        if k + 1 < esteps:
            with torch.cuda.stream(copy):      # next step's input, during this step
                d_dev[j].copy_(d_host, non_blocking=True)
                h2d[j].record(copy)
        main.wait_event(h2d[i])
        if k >= 2:
            main.wait_event(d2h[i])            # buffer set i's results are home
        plan.realize(d_dev[i], seeds(1000 + k), tol, out=out_dev[i])
        done[i].record(main)
        with torch.cuda.stream(copy):
            copy.wait_event(done[i])
            out_host[i].copy_(out_dev[i], non_blocking=True)
            d2h[i].record(copy)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / esteps
    e2e = {"value": B * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": d_host.numel() * esz,
           "d2h_bytes_per_step": out_host[0].numel() * esz}

    # Lanczos estimate of the preconditioned operator's spectrum from the CG
    # coefficients of the last realization (Sect. 6.4)
    t0 = time.perf_counter()
    lz = plan.lanczos(0)
    lanczos = {"lmin": lz["lmin"], "lmax": lz["lmax"], "kappa": lz["kappa"],
               "iterations": int(len(lz["alpha"])),
               "ms": (time.perf_counter() - t0) * 1e3}

    # kernel relaxation (Sect. 5, eq. Algo) on the same workload: sweeps/s
    torch.cuda.synchronize()
    rsweeps = 20
    t0 = time.perf_counter()
    _, rst = plan.relax(d, rsweeps)
    relax = {"sweeps": rsweeps, "ms_per_sweep": (time.perf_counter() - t0) * 1e3 / rsweeps,
             "rel_resid": rst[0]["rel_resid"], "batch": B}

    strip_meas = strips_measurement() if (rank == 0 and not args.no_strips) else None
    far = far_interior_measurement() if (rank == 0 and not args.no_strips) else None
    lms = laplace_ms_measurement() if (rank == 0 and not args.no_strips) else None
    act = act_measurement() if (rank == 0 and not args.no_strips) else None

    # roofline of the hot-loop passes (CUDA events on the plan's stream)
    peaks, peak_src = measured_peaks()
    passes = {0: ("k_col (column FFT, x 1/(nP), inverse FFT)", 3),
              1: ("k_row src (r, u update + R2C)", 1),
              2: ("k_row src (p update + R2C)", 1),
              3: ("k_row sink (C2R + q = P_x, p^T q)", 2),
              4: ("k_row mid (C2R, P_x, R2C)", 1)}
    timing = {}
    for pid, (name, per_iter) in passes.items():
        pms, pbytes = plan.time_pass(pid, reps=20)
        timing[pid] = (name, per_iter, pms, pbytes)
    dom = max(timing, key=lambda k: timing[k][1] * timing[k][2])
    name, _, pms, pbytes = timing[dom]
    achieved = pbytes / (pms / 1e3) / 1e9
    traffic = None
    if name in TRAFFIC and mode in ("fp32", "mixed") and \
            kernel_src_hash() == TRAFFIC["src_hash"] and (ny, nx) == (4096, 4096):
        per_inst, shared = TRAFFIC[name]
        traffic = (per_inst * B + shared) * 1e6
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": f"{peak_src} (hbm_gbs, burst)",
                "bytes_per_launch": pbytes, "ms_per_launch": pms}
    pass_table = {timing[k][0]: {"ms": round(timing[k][2], 4),
                                 "GB/s": round(timing[k][3] / timing[k][2] / 1e6, 1),
                                 "per_iter": timing[k][1]} for k in timing}
    plan.close()

    # plain FP64 GPU PCG on the same inputs
    fp64 = None
    if not args.no_fp64 and args.fp64_steps > 0 and mode != "fp64":
        p64 = cg.Plan(P, obs, mode="fp64", batch=B)
        d64 = d.to(torch.float64)
        p64.realize(d64, seeds(0), tol)
        torch.cuda.synchronize()
        e0.record(stream)
        it64 = 0
        for k in range(args.fp64_steps):
            _, st = p64.realize(d64, seeds(1 + k), tol)
            it64 += sum(s["iters"] for s in st)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        fp64 = {"value": B * args.fp64_steps / (ms64 / 1e3), "unit": UNIT,
                "ms_per_step": ms64 / args.fp64_steps,
                "cg_iters_per_s": it64 / (ms64 / 1e3),
                "iters_per_realization": it64 / (B * args.fp64_steps)}
        p64.close()

    # cuFFT-based PCG (timed comparison, not part of the library), and the
    # library's FP32 mode at the cuFFT FP32 arm's tolerance
    cufft = cufft_arm(P, obs, d, B, tol) if (rank == 0 and not args.no_fp64) else None
    if cufft is not None:
        p32 = cg.Plan(P, obs, mode="fp32", batch=B)
        d32 = d.float().contiguous()
        ms32, (_, st32) = _events_ms(lambda: p32.realize(d32, seeds(0), 1e-5), 1)
        cufft["library_fp32_same_tol"] = {"realizations_per_s": B / (ms32 / 1e3), "ms_per_step": ms32,
                                          "batch": B, "tol": 1e-5,
                                          "iters_per_realization": sum(x["iters"] for x in st32) / B}
        p32.close()
        del d32
        torch.cuda.empty_cache()

    configs, keep = (None, None)
    if rank == 0 and not args.no_configs:
        configs, keep = configs_measurement()

    cpu, oracle_err = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        import numpy as np
        import oracle as O
        dn = d.cpu().numpy().astype("float64")
        cpu_iters = 3
        setup, t_iter = oracle_sample(P, obs, dn, spec["seeds"][0], cpu_iters)
        n_it = fp64["iters_per_realization"] if fp64 else FP64_ITERS_WIDE4096
        cpu = {"value": 1.0 / (setup + n_it * t_iter), "unit": UNIT, "cores": threads_used(),
               "kind": "oracle",
               "sample": (f"FP64 oracle (own C FFT on {threads_used()} host threads, NumPy "
                          f"element-wise) on the full {ny}x{nx} workload: draw + RHS "
                          f"({setup:.1f} s) and {cpu_iters} preconditioned CG iterations "
                          f"({t_iter:.2f} s each), scaled to the {n_it:.1f} iterations per "
                          f"realization the FP64 GPU PCG needed in this run")}
        # error of the headline's last realization against the oracle
        x_last = last_x.double().cpu().numpy()
        oracle_err = oracle_check(P, obs, dn, x_last, last_seed, tol)
        # whole realizations on the host cores, checked against the GPU's
        if keep is not None:
            for name in ("plain64", "patch1024"):
                Pk, obsk, dk, xk, seedk, tolk = keep[name]
                t0 = time.perf_counter()
                ref = O.realize(Pk, obsk, dk, seedk, tol=tolk)
                sec = time.perf_counter() - t0
                mk = obsk == 0
                configs[name]["cpu_baseline"] = {
                    "value": 1.0 / sec, "unit": UNIT, "cores": threads_used(), "kind": "oracle",
                    "sample": f"one whole realization ({ref.pcg.iters} iterations)"}
                configs[name]["rel_err_vs_oracle_same_tol"] = float(
                    np.linalg.norm(xk[mk] - ref.x[mk]) / np.linalg.norm(ref.x[mk]))
                configs[name]["observed_bit_exact"] = bool(np.array_equal(xk[~mk], dk[~mk]))
        if act is not None:   # the same oracle sample on the Sect. 3 map
            a_out, aP, aobs, ad, aspec = act
            setup, t_iter = oracle_sample(aP, aobs, ad.cpu().numpy().astype("float64"),
                                          aspec["seeds"][0], 1)
            n_it = a_out["precond"]["iters_per_realization"]
            a_out["precond"]["cpu_baseline"] = {
                "value": 1.0 / (setup + n_it * t_iter), "unit": UNIT, "cores": threads_used(),
                "kind": "oracle",
                "sample": (f"draw + RHS ({setup:.1f} s) and 1 preconditioned CG iteration "
                           f"({t_iter:.2f} s), scaled to {n_it:.0f} iterations")}

    if rank == 0:
        metric = METRIC if args.workload == "wide4096" else \
            f"constrained realizations/s at {ny}x{nx} ({args.workload}, refined to {tol:g})"
        line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"mixed": "f32+df64", "fp32": "f32", "fp64": "f64"}[mode],
                "data": "synthetic",
                "config": workload_config(args.workload, (ny, nx), B, tol, mode,
                                          (obs == 0).mean(), world,
                                          loops="host" if args.host_loops else "graph",
                                          update_delta=args.update_delta),
                "cg_iters_per_s": iters_per_s,
                "iters_per_realization": iters / (B * args.steps),
                "worst_true_rel_resid": worst_resid,
                "fp64_pcg": fp64,
                "cufft_pcg": cufft,
                "speedup_vs_fp64": (value / world / fp64["value"]) if fp64 else None,
                "gpu_launches": launches, "e2e": e2e, "roofline": roofline,
                "passes": pass_table, "lanczos": lanczos, "relax": relax, "strips": strip_meas,
                "far_interior": far, "laplace_ms": lms,
                "act7000x600": act[0] if act is not None else None,
                "configs": configs,
                "oracle_check": oracle_err,
                "clocks": clk.summary(),
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
