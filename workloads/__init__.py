"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only builds input arrays (power spectra on the Fourier grid,
observation masks, band-power templates).  It contains none of the fill-in
method's arithmetic: no transforms, no solves, no random-field draws.
"""
from .synth import (  # noqa: F401
    kgrid_half,
    spectrum_lorentz_beam,
    spectrum_cmb_like,
    spectrum_cmb_bands,
    band_index_half,
    band_templates_half,
    band_mask_rows,
    add_discs,
    mask_band_discs,
    mask_area_target,
    WORKLOADS,
    workload,
)
