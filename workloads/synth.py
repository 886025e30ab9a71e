"""Synthetic spectra, masks and band templates for the flat periodic sky.

Conventions (shared by every consumer):

* A map is a real ``ny x nx`` array on a periodic grid with unit pixel size.
* Fourier modes are ``k = 2*pi*m/N`` with ``m`` in ``[-N/2, N/2)`` along each
  axis, so the Nyquist mode has ``|k| = pi``.  Spectra are handed out on the
  half plane ``ny x (nx//2 + 1)`` in the row-major layout of a real 2D FFT
  (row index ``my``, column index ``mx >= 0``).
* ``observed[i] = 1`` marks a pixel whose value is known (a constraint);
  ``observed[i] = 0`` marks a masked pixel that the method fills in.

The spectrum shapes stand in for the paper's ACT-like model
``P_l = w_l C_l + N_l`` (Sect. 3): a beam window on a red signal spectrum plus
a white-noise floor.  Masks stand in for the paper's point-source holes and
Galactic cut (Sect. 3): a full-width band of rows plus discs.  All random
choices come from NumPy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# Fourier grid and spectra
# ---------------------------------------------------------------------------

def kgrid_half(ny: int, nx: int) -> np.ndarray:
    """|k| on the half plane ``ny x (nx//2+1)`` (float64)."""
    my = np.fft.fftfreq(ny) * ny          # 0..ny/2-1, -ny/2..-1
    mx = np.arange(nx // 2 + 1, dtype=np.float64)
    ky = TWO_PI * my / ny
    kx = TWO_PI * mx / nx
    return np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)


def spectrum_lorentz_beam(ny: int, nx: int, k0: float = TWO_PI / 32.0,
                          sb: float = 1.5, noise_frac: float = 1e-4) -> np.ndarray:
    """``P(k) = exp(-k^2 sb^2) / (k^2 + k0^2) + N`` with ``N = noise_frac * S(k0)``.

    ``S(k0)`` is the signal part (beam included) evaluated at ``k = k0``.
    """
    k = kgrid_half(ny, nx)
    signal = np.exp(-(k * sb) ** 2) / (k * k + k0 * k0)
    s_k0 = math.exp(-(k0 * sb) ** 2) / (2.0 * k0 * k0)
    return signal + noise_frac * s_k0


def _cmb_signal(k: np.ndarray, k_lo: float, sb: float, k_peak: float,
                k_d: float) -> np.ndarray:
    """Red (k^-2) below ``k_peak``, flat above, damped and beamed."""
    kk = np.maximum(k, k_lo)
    red = np.where(kk < k_peak, (k_peak / kk) ** 2, 1.0)
    return red * np.exp(-(k / k_d) ** 2) * np.exp(-(k * sb) ** 2)


CMB_K_PEAK = TWO_PI / 200.0
CMB_K_DAMP = TWO_PI / 24.0


def cmb_noise_level(k_lo: float, sb: float = 2.0, k_peak: float = CMB_K_PEAK,
                    k_d: float = CMB_K_DAMP, noise_frac: float = 1e-3) -> float:
    """White-noise floor ``N = noise_frac * S(k_d)``."""
    return float(noise_frac * _cmb_signal(np.array(k_d), k_lo, sb, k_peak, k_d))


def spectrum_cmb_like(ny: int, nx: int, k_lo: float, sb: float = 2.0,
                      k_peak: float = CMB_K_PEAK, k_d: float = CMB_K_DAMP,
                      noise_frac: float = 1e-3) -> np.ndarray:
    """CMB-like ``P(k) = S(k) + N`` on the half plane.

    ``S(k) = (k_peak / max(k, k_lo))^2`` for ``k < k_peak`` and 1 above, times
    ``exp(-(k/k_d)^2) exp(-k^2 sb^2)``; ``N = noise_frac * S(k_d)``.
    """
    k = kgrid_half(ny, nx)
    return _cmb_signal(k, k_lo, sb, k_peak, k_d) + cmb_noise_level(
        k_lo, sb, k_peak, k_d, noise_frac)


def band_edges(k_lo: float, nbands: int = 32) -> np.ndarray:
    """``nbands + 1`` log-spaced edges from ``k_lo`` to ``pi*sqrt(2)``."""
    return np.geomspace(k_lo, math.pi * math.sqrt(2.0), nbands + 1)


def band_index_half(ny: int, nx: int, k_lo: float, nbands: int = 32) -> np.ndarray:
    """Band number (int32) of every half-plane mode; modes below ``k_lo``
    (including k = 0) belong to band 0."""
    k = kgrid_half(ny, nx)
    b = np.searchsorted(band_edges(k_lo, nbands), k, side="right") - 1
    return np.clip(b, 0, nbands - 1).astype(np.int32)


def band_templates_half(ny: int, nx: int, k_lo: float, nbands: int = 32,
                        sb: float = 2.0):
    """Signal templates ``T_b(k) = 1[k in b] S(k)`` as (band index, S, N)."""
    k = kgrid_half(ny, nx)
    sig = _cmb_signal(k, k_lo, sb, CMB_K_PEAK, CMB_K_DAMP)
    return band_index_half(ny, nx, k_lo, nbands), sig, cmb_noise_level(k_lo, sb)


def spectrum_cmb_bands(ny: int, nx: int, amps: np.ndarray, k_lo: float,
                       sb: float = 2.0) -> np.ndarray:
    """``P(k) = sum_b a_b 1[k in b] S(k) + N``; equals the CMB-like spectrum
    when every amplitude is 1."""
    amps = np.asarray(amps, dtype=np.float64)
    bidx, sig, noise = band_templates_half(ny, nx, k_lo, len(amps), sb)
    return amps[bidx] * sig + noise


# ---------------------------------------------------------------------------
# Masks
# ---------------------------------------------------------------------------

def band_mask_rows(ny: int, nx: int, nrows: int) -> np.ndarray:
    """Boolean masked-pixel map with ``nrows`` full-width rows centred at ny/2."""
    masked = np.zeros((ny, nx), dtype=bool)
    if nrows > 0:
        r0 = ny // 2 - nrows // 2
        masked[r0:r0 + nrows, :] = True
    return masked


def add_discs(masked: np.ndarray, centres: np.ndarray, radii: np.ndarray) -> None:
    """Mask every pixel within (periodic, minimum-image) distance ``r`` of a
    disc centre.  Centres are continuous positions ``(cy, cx)`` in pixels."""
    ny, nx = masked.shape
    for (cy, cx), r in zip(centres, radii):
        iy = np.arange(int(math.floor(cy - r)) - 1, int(math.ceil(cy + r)) + 2)
        ix = np.arange(int(math.floor(cx - r)) - 1, int(math.ceil(cx + r)) + 2)
        dy = (iy - cy + ny / 2.0) % ny - ny / 2.0
        dx = (ix - cx + nx / 2.0) % nx - nx / 2.0
        inside = dy[:, None] ** 2 + dx[None, :] ** 2 <= r * r
        yy, xx = np.nonzero(inside)
        masked[iy[yy] % ny, ix[xx] % nx] = True


def mask_band_discs(ny: int, nx: int, band_rows: int, ndiscs: int,
                    rmin: float, rmax: float, seed: int) -> np.ndarray:
    """``observed`` (uint8, 1 = observed) for a band of rows plus discs with
    radius uniform in ``[rmin, rmax]`` at uniform random centres."""
    rng = np.random.Generator(np.random.PCG64(seed))
    masked = band_mask_rows(ny, nx, band_rows)
    centres = rng.uniform(0.0, 1.0, size=(ndiscs, 2)) * np.array([ny, nx])
    radii = rng.uniform(rmin, rmax, size=ndiscs) if rmax > rmin else np.full(ndiscs, rmin)
    add_discs(masked, centres, radii)
    return (~masked).astype(np.uint8)


def mask_area_target(ny: int, nx: int, seed: int, amin: float = 0.05,
                     amax: float = 0.25, band_share: float = 0.7,
                     rmin: float = 2.0, rmax: float = 12.0) -> np.ndarray:
    """Band-plus-discs mask whose masked area reaches a target ``a ~ U(amin, amax)``.

    The band takes ``band_share * a`` of the rows; discs (radius ~ U(rmin, rmax))
    are added one at a time until the masked fraction reaches ``a``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.uniform(amin, amax)
    masked = band_mask_rows(ny, nx, int(round(band_share * a * ny)))
    target = a * ny * nx
    while masked.sum() < target:
        c = rng.uniform(0.0, 1.0, size=(1, 2)) * np.array([ny, nx])
        add_discs(masked, c, rng.uniform(rmin, rmax, size=1))
    return (~masked).astype(np.uint8)


# ---------------------------------------------------------------------------
# Named workloads (sizes and recipes of the five measured configurations)
# ---------------------------------------------------------------------------

WORKLOADS = {
    # Plain method in FP64 on a 64x64 torus, one realization, CG tol 1e-8.
    "plain64": dict(ny=64, nx=64, spectrum="lorentz", band_rows=8, ndiscs=5,
                    rmin=3.0, rmax=3.0, mask_seed=11, data_seed=1, seeds=[2],
                    tol=1e-8, precision="fp64"),
    # 1024^2 patch, FP32 operator with FP64-accurate reductions, tol 1e-6.
    "patch1024": dict(ny=1024, nx=1024, spectrum="cmb", k_lo_n=1024,
                      band_frac=0.10, ndiscs=200, rmin=2.0, rmax=12.0,
                      mask_seed=12, data_seed=3, seeds=[4], tol=1e-6,
                      precision="fp32"),
    # 256 realizations at 256^2 / 512^2 / 1024^2 (128 / 96 / 32), own masks.
    "batch_mixed": dict(sizes=[(256, 128), (512, 96), (1024, 32)],
                        spectrum="cmb", k_lo_n=1024, mask_seed=13,
                        data_seed=5, seed0=1000, tol=1e-6, precision="fp32"),
    # 2048^2 differentiation case with 32 log-spaced band powers.
    "grad2048": dict(ny=2048, nx=2048, spectrum="cmb", k_lo_n=2048,
                     band_frac=0.15, ndiscs=500, rmin=2.0, rmax=12.0,
                     mask_seed=14, data_seed=6, seeds=[7], tol=1e-6,
                     nbands=32, precision="fp32"),
    # The flat-sky season map of Sect. 3: 7000 x 600 pixels (about 0.5 arcmin,
    # 300 square degrees) with about 400 point-source holes of 0.01 square
    # degrees (radius about 6.7 pixels) and no band; a mixed-radix grid
    # (nx/2 = 3500 = 2^2 5^3 7, ny = 600 = 2^3 3 5^2).  Batch of 4 (the
    # four simulated maps), mixed precision refined to 1e-10.
    "act7000x600": dict(ny=600, nx=7000, spectrum="cmb", k_lo_n=4096,
                        band_frac=0.0, ndiscs=400, rmin=6.7, rmax=6.7,
                        mask_seed=16, data_seed=9, seeds=list(range(200, 204)),
                        tol=1e-10, precision="mixed"),
    # 4096^2 wide cut, batch of 8, refined to a relative residual of 1e-10.
    "wide4096": dict(ny=4096, nx=4096, spectrum="cmb", k_lo_n=4096,
                     band_frac=0.20, ndiscs=2000, rmin=2.0, rmax=20.0,
                     mask_seed=15, data_seed=8, seeds=list(range(100, 108)),
                     tol=1e-10, precision="mixed"),
}


def workload(name: str, scale: int = 1):
    """Build ``(P_half, observed, spec)`` for a single-grid workload.

    ``scale`` > 1 shrinks the grid by that factor (disc radii, band fraction
    and spectrum shape in physical units are kept) for fast parity cases.
    """
    spec = dict(WORKLOADS[name])
    ny, nx = spec["ny"] // scale, spec["nx"] // scale
    if spec["spectrum"] == "lorentz":
        P = spectrum_lorentz_beam(ny, nx)
        band_rows = spec["band_rows"] // scale
    else:
        k_lo = TWO_PI / spec["k_lo_n"]
        P = spectrum_cmb_like(ny, nx, k_lo)
        spec["k_lo"] = k_lo
        band_rows = int(round(spec["band_frac"] * ny))
    ndiscs = max(1, spec["ndiscs"] // (scale * scale))
    observed = mask_band_discs(ny, nx, band_rows, ndiscs, spec["rmin"],
                               spec["rmax"], spec["mask_seed"])
    spec.update(ny=ny, nx=nx, band_rows=band_rows, ndiscs=ndiscs)
    return P, observed, spec
