"""Laplace interpolation into a masked region: the exact discrete solve, the
far-interior test of Sect. 6.1, and the kernel-based solver of Sect. 6.3.

The discrete Laplace equation on the masked pixels with the map outside as
Dirichlet data is the maximum-likelihood fill for the spectrum
``P = 1/(lambda(k) + m^2)``, ``lambda = 4 sin^2(k_x/2) + 4 sin^2(k_y/2)`` (the
5-point stencil) as ``m -> 0``: the precision operator is ``-Delta + m^2``, and
``(C^-1 x)_M = 0`` is the stencil equation on M.  On a periodic band this is
the discrete counterpart of the sinh interpolation of Sect. 6.1.  The solve is
``fill_ml`` on a plan for that spectrum; this module only builds the inputs
and sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import Plan, fill_subdivide


def stencil_spectrum(ny, nx, m2=1e-8):
    """``1 / (lambda(k) + m^2)`` on the half plane ``ny x (nx/2 + 1)``."""
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)
    kx = 2.0 * np.pi * np.arange(nx // 2 + 1) / nx
    lam = 4.0 * np.sin(ky[:, None] / 2.0) ** 2 + 4.0 * np.sin(kx[None, :] / 2.0) ** 2
    return 1.0 / (lam + m2)


def laplace_fill(observed, x, mode="mixed", tol=1e-10, max_iter=20000, m2=1e-8):
    """Harmonic (5-point stencil) interpolation of the device map ``x`` into
    the pixels where ``observed`` is 0.  Returns ``(map, stats)``."""
    ny, nx = observed.shape
    plan = Plan(stencil_spectrum(ny, nx, m2), np.ascontiguousarray(observed, dtype=np.uint8),
                mode=mode, max_iter=max_iter)
    out, st = plan.ml(x, tol)
    plan.close()
    return out[0], st[0]


def band_rows(ny, nx, rows):
    """``observed`` map (uint8) of a band of ``rows`` full-width rows centred at ny/2."""
    obs = np.ones((ny, nx), dtype=np.uint8)
    y0 = ny // 2 - rows // 2
    obs[y0:y0 + rows] = 0
    return obs


def far_interior(P_half, d, rows, layer, mode="mixed", tol=1e-8):
    """Sect. 6.1's test: the exact ML fill of a band of ``rows`` rows, then the
    Laplace interpolation into the band's interior after removing ``layer``
    rows along each boundary, from the ML values there.  Returns the Laplace
    map, the ML map, the inner band's observed map and solver stats."""
    ny, nx = d.shape
    outer = band_rows(ny, nx, rows)
    inner = band_rows(ny, nx, rows - 2 * layer)
    plan = Plan(P_half, outer, mode=mode)
    ml, st_ml = plan.ml(d, tol)
    plan.close()
    lap, st_lap = laplace_fill(inner, ml[0], mode=mode)
    return lap, ml[0], inner, (st_ml[0], st_lap)


def ms_radii(nk=9, rho0=1.5, q=1.55):
    """The Sect. 6.3 solver's annuli ``(r_in, r_out)``: centre radii
    ``rho0 q^j`` in geometric progression, bounds at the geometric midpoints
    (consecutive annuli tile the plane), the smallest solid (the centre pixel
    excluded: the eight neighbours)."""
    out = []
    for j in range(nk):
        rho = rho0 * q ** j
        out.append((0.0 if j == 0 else rho / np.sqrt(q), rho * np.sqrt(q)))
    return out


def ms_classes(obs_dev, radii):
    """Annulus index of every masked pixel (device uint8 map): the largest
    ``j`` whose disc of radius ``r_out_j`` holds no observed pixel (the Sect.
    6.2 layer of width ``2 r_out_j`` at threshold 0 does not contain it), else
    0: the thin layer along the boundary, where the smallest annulus reaches
    the observed region."""
    import torch
    obs = obs_dev.cpu().numpy().astype(bool)
    cls = np.zeros(obs.shape, dtype=np.uint8)
    for j, (_, r_out) in enumerate(radii):
        layer = fill_subdivide(obs_dev, 2.0 * r_out, 0.0).cpu().numpy().astype(bool)
        cls[~obs & ~layer] = j
    return torch.from_numpy(cls).to(obs_dev.device)


def laplace_ms(observed, d, iters, radii=None, mode="mixed"):
    """``iters`` sweeps of the kernel-based Laplace solver of Sect. 6.3 on the
    device map ``d`` (values on the mask ignored; the sweeps start from 0
    there).  Returns ``(map, stats)``."""
    import torch
    radii = ms_radii() if radii is None else radii
    observed = np.ascontiguousarray(observed, dtype=np.uint8)
    ny, nx = observed.shape
    plan = Plan(np.ones((ny, nx // 2 + 1)), observed, mode=mode)
    plan.set_annuli([r[0] for r in radii], [r[1] for r in radii])
    cls = ms_classes(torch.from_numpy(observed).to(d.device), radii)
    out, st = plan.laplace_ms(d.to(plan.dtype).contiguous(), iters, cls)
    plan.close()
    return out[0], st[0]
