"""CPU-only checks of the boundary: the C-ABI library builds, loads without a
GPU and exports every function ``include/cgfill.h`` declares; the Python
binding mirrors those names; no compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1109_0286_gb300 as cg
from paper_1109_0286_gb300 import _build
from workloads import synth, workload, WORKLOADS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cgfill.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fill_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return cg.load()


def test_header_and_binding_agree():
    assert declared_functions() == sorted(cg.EXPORTED_SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert callable(getattr(lib, name))


def test_host_only_calls(lib):
    o = cg.fill_opts_default()
    assert (o.mode, o.precond, o.batch, o.max_iter, o.max_refine) == (2, 1, 1, 10000, 10)
    assert o.inner_tol == 1e-6 and o.update_delta == 1e-2
    assert cg.fill_version() == 1
    assert cg.fill_strerror(0) == "ok"
    assert "converged" in cg.fill_strerror(3)
    # argument validation happens before any device work (nx / 2 = 22 = 2 x 11:
    # neither a power of two nor a product of 2, 3, 5, 7)
    plan = ctypes.c_void_p()
    P = np.ones((64, 33))
    m = np.ones((64, 64), np.uint8)
    st = lib.fill_init(ctypes.byref(plan), 64, 44, P.ctypes.data, m.ctypes.data,
                       ctypes.byref(o), None)
    assert st == 1 and not plan.value
    # sizes neither power-of-two nor mixed-radix-valid: odd nx, a prime factor
    # above 7, nx/2 or ny above 4096, ny below 8
    big, mbig = np.ones(400_000), np.ones(700_000, np.uint8)   # cover ny * nx of every case
    for ny, nx in ((60, 85), (66, 84), (60, 86), (8200, 84), (60, 8400), (6, 84), (4, 64)):
        st = lib.fill_init(ctypes.byref(plan), ny, nx, big.ctypes.data, mbig.ctypes.data,
                           ctypes.byref(o), None)
        assert st == 1 and not plan.value, (ny, nx)
    assert lib.fill_realize(None, None, 0, None, 1e-6, None, None) == 1
    # option ranges are checked before any device work (lanes: 0..8)
    Pv, mv = np.ones((64, 33)), np.ones((64, 64), np.uint8)
    for field, bad in (("lanes", 9), ("lanes", -1), ("col_kernel", 2), ("host_loops", 2)):
        ob = cg.fill_opts_default()
        setattr(ob, field, bad)
        st = lib.fill_init(ctypes.byref(plan), 64, 64, Pv.ctypes.data, mv.ctypes.data,
                           ctypes.byref(ob), None)
        assert st == 1 and not plan.value, field
    lib.fill_destroy(None)


def test_struct_layouts(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler
    gives the header's structs."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    fields = [f for f, _ in cg.FillOpts._fields_]
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "cgfill.h"\nint main(void) {\n'
        '  printf("%zu %zu\\n", sizeof(fill_opts), sizeof(fill_stats));\n'
        + "".join(f'  printf("%zu\\n", offsetof(fill_opts, {f}));\n' for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(cg.FillOpts)
    assert int(out[1]) == ctypes.sizeof(cg.FillStats)
    for f, off in zip(fields, out[2:]):
        assert getattr(cg.FillOpts, f).offset == int(off), f


def test_mask_generators():
    obs = synth.mask_band_discs(256, 256, 26, 20, 2.0, 12.0, seed=3)
    assert obs.dtype == np.uint8 and set(np.unique(obs)) <= {0, 1}
    assert np.all(obs[128 - 13:128 + 13] == 0)
    # periodic discs wrap around the edges
    m = np.zeros((32, 32), bool)
    synth.add_discs(m, np.array([[0.0, 0.0]]), np.array([2.5]))
    assert m[0, 0] and m[31, 31] and m[0, 30] and not m[16, 16]
    for s in range(5):
        a = 1 - synth.mask_area_target(256, 256, seed=s).mean()
        assert 0.05 <= a <= 0.27


def test_spectra_hermitian_and_positive():
    for ny, nx in [(64, 64), (32, 128)]:
        for P in (synth.spectrum_lorentz_beam(ny, nx),
                  synth.spectrum_cmb_like(ny, nx, 2 * np.pi / 1024)):
            assert P.shape == (ny, nx // 2 + 1) and np.all(P > 0)
            my = (-np.arange(ny)) % ny
            assert np.array_equal(P[:, 0], P[my, 0]) and np.array_equal(P[:, -1], P[my, -1])
    k_lo = 2 * np.pi / 256
    amps = np.ones(32)
    assert np.allclose(synth.spectrum_cmb_bands(256, 256, amps, k_lo),
                       synth.spectrum_cmb_like(256, 256, k_lo), rtol=1e-15)
    b = synth.band_index_half(256, 256, k_lo)
    assert b[0, 0] == 0 and b.max() == 31


def test_workload_table():
    assert set(WORKLOADS) == {"plain64", "patch1024", "batch_mixed", "grad2048", "wide4096",
                              "act7000x600"}
    sizes = WORKLOADS["batch_mixed"]["sizes"]
    assert sum(c for _, c in sizes) == 256
    # the Sect. 3 season map: 7000 x 600, ~400 holes of 0.01 deg^2 (~141 pixels
    # of 0.5 arcmin); nx/2 = 3500 = 2^2 5^3 7, ny = 600 = 2^3 3 5^2
    _, obs, spec = workload("act7000x600")
    assert obs.shape == (600, 7000) and spec["ndiscs"] == 400
    assert 0.8 * 400 * 141 <= int((obs == 0).sum()) <= 400 * 141 * 1.05


def test_laplace_radii_match_the_oracle():
    """The package's annulus radii (used by the bench and the wrapper) are the
    oracle's reading of the Sect. 6.3 kernels."""
    import oracle as O
    from paper_1109_0286_gb300 import laplace
    for nk in (1, 5, 9, 13):
        assert np.allclose(laplace.ms_radii(nk), O.ms_radii(nk), rtol=1e-15, atol=0)


def test_profile_summaries_are_text_with_their_commands():
    """Every ncu summary under profiles/ is short text naming the command that
    made it, with the clocks left alone (--clock-control none)."""
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")
    names = sorted(os.listdir(root))
    assert names and all(n.endswith((".md", ".txt")) for n in names)
    for n in names:
        text = open(os.path.join(root, n)).read()
        assert len(text) < 16384, n
        assert "ncu " in text and "--clock-control none" in text, n


@pytest.mark.parametrize("ny,nx,precond", [(32, 48, True), (24, 32, False)])
def test_cufft_comparison_arm_computes_the_realization(ny, nx, precond):
    """The bench's cuFFT comparison (PyTorch FFT, here on the CPU) computes
    the same constrained realization as the oracle from the same draw."""
    import sys
    import torch
    import oracle as O
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    P = synth.spectrum_cmb_like(ny, nx, 2 * np.pi / nx)
    obs = synth.mask_band_discs(ny, nx, 5, 2, 2.0, 3.0, 4)
    Pf = O.hermitian_full(P, nx)
    d = O.draw(Pf, 7)
    y = O.draw(Pf, 11)
    x, it = bench.cufft_pcg_realize(torch.from_numpy(P), torch.from_numpy(obs == 0),
                                    torch.from_numpy(d), torch.from_numpy(y)[None], 1e-12,
                                    precond=precond)
    ref = O.realize(P, obs, d, 11, tol=1e-13, precond=precond)
    m = obs == 0
    got = x[0].numpy()
    assert np.array_equal(got[~m], d[~m]) and it > 0
    assert np.linalg.norm(got[m] - ref.x[m]) <= 1e-9 * np.linalg.norm(ref.x[m])


def test_static_apply_rejections_need_no_gpu(lib):
    """fill_apply_static validates its arguments before any CUDA call and
    records the reason (fill_last_error) on every rejection."""
    P = np.ones((64, 33))
    x = np.zeros((64, 64), np.float32)
    y = np.zeros((64, 64), np.float32)
    m = np.ones((64, 64), np.uint8)
    cases = [
        ((64, 64, P.ctypes.data, m.ctypes.data, 7, x.ctypes.data, y.ctypes.data, None), "which"),
        ((64, 64, P.ctypes.data, None, 2, x.ctypes.data, y.ctypes.data, None), "mask"),
        ((64, 64, P.ctypes.data, m.ctypes.data, 0, x.ctypes.data, x.ctypes.data, None), "alias"),
        ((64, 60, P.ctypes.data, m.ctypes.data, 0, x.ctypes.data, y.ctypes.data, None), "powers of two"),
        ((2048, 2048, P.ctypes.data, m.ctypes.data, 0, x.ctypes.data, y.ctypes.data, None), "too large"),
        ((64, 64, None, m.ctypes.data, 0, x.ctypes.data, y.ctypes.data, None), "null"),
    ]
    for args, why in cases:
        assert lib.fill_apply_static(*args) == 1
        assert why in cg.fill_last_error(), (why, cg.fill_last_error())


def test_new_entry_points_reject_bad_arguments_on_the_host(lib):
    """fill_set_spectrum and fill_realize_batch check their arguments before
    touching a plan or the device."""
    P = np.ones((64, 33))
    assert lib.fill_set_spectrum(None, P.ctypes.data) == 1
    assert lib.fill_realize_batch(None, 1, None, None, 1e-6, None, None) == 1
    plans = (ctypes.c_void_p * 1)(None)
    assert lib.fill_realize_batch(plans, 0, None, None, 1e-6, None, None) == 1


def test_band_power_spectrum_model():
    """P(k) = sum_b a_b 1[band(k) = b] S(k) + N, the parameterisation the
    autograd wrapper hands to fill_set_spectrum."""
    k_lo = 2 * np.pi / 64
    bidx, sig, noise = synth.band_templates_half(64, 64, k_lo, 8)
    model = cg.BandPowerSpectrum(bidx, sig, noise)
    a = np.linspace(0.5, 1.5, 8)
    assert np.allclose(model(np.ones(8)), synth.spectrum_cmb_like(64, 64, k_lo), rtol=1e-14)
    assert np.array_equal(model(a), a[bidx] * sig + noise)
    with pytest.raises(ValueError):
        model(np.ones(7))
