"""Noise-boosted strip refinement (Sect. 6.4) on the periodic grid.

The map is refined across nested strips of the mask, each refilled with the
maximum-likelihood solution for a boosted-noise spectrum ``P = S + beta N``
while the current map outside the strip acts as data.  The strips come from
the subdivision of Sect. 6.2 (``fill_subdivide``), every solve from
``fill_ml`` on a plan for that strip; this module only sequences the C-ABI
calls.
"""
from __future__ import annotations

import numpy as np

from . import Plan, fill_subdivide

# (noise boost beta, strip width w in pixels) used in Sect. 6.4
PAPER_STAGES = ((2000.0, 100.0), (400.0, 35.0), (40.0, 15.0), (1.0, 7.0))


def strip_refine(S_half, N_half, observed, d, stages=PAPER_STAGES, mode="fp64", tol=1e-8,
                 max_iter=10000, start_sweeps=0):
    """Refine a fill of data ``d`` (device map; values on the mask ignored)
    across the strips of ``stages``.  The start map is ``d`` on the observed
    pixels and, on the mask, 0 relaxed by ``start_sweeps`` sweeps of the
    kernel relaxation of Sect. 5 (``fill_relax``).  Returns ``(x, stats)``
    with one entry per stage: ``(beta, w, strip pixels, CG iterations)``."""
    import torch
    S_half = np.asarray(S_half, dtype=np.float64)
    N_half = np.asarray(N_half, dtype=np.float64)
    observed = np.ascontiguousarray(observed, dtype=np.uint8)
    obs_dev = torch.from_numpy(observed).to(d.device)
    base = Plan(S_half + N_half, observed, mode=mode, max_iter=max_iter)
    x, _ = base.relax(d, start_sweeps)
    base.close()
    x = x[0]
    log = []
    for beta, w in stages:
        layer = fill_subdivide(obs_dev, w).cpu().numpy()
        npx = int(layer.sum())
        if npx == 0:
            log.append((beta, w, 0, 0))
            continue
        strip_obs = (1 - layer).astype(np.uint8)
        plan = Plan(S_half + beta * N_half, strip_obs, mode=mode, max_iter=max_iter)
        out, st = plan.ml(x, tol)
        plan.close()
        x = out[0]
        log.append((beta, w, npx, st[0]["iters"]))
    return x, log
