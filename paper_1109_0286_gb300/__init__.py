"""GB300 constrained-realization fill-in of masked pixels on the flat sky.

Python binding of the C ABI declared in ``include/cgfill.h`` (Bucher & Louis,
arXiv:1109.0286, Sects. 2.1-2.4 on the periodic flat domain of Sect. 3).  The
functions below only marshal arguments: every numerical step runs in the CUDA
kernels of ``libcgfill.so``.  There is no CPU fallback; using the library
without the built extension or without a GPU raises.

Low-level names mirror the C ABI (``fill_init``, ``fill_realize``,
``fill_realize_batch``, ``fill_set_spectrum``, ``fill_draw``, ``fill_apply``,
``fill_history``, ``fill_destroy``, ``fill_strerror``, ``fill_version``);
``Plan`` wraps them for torch tensors, and ``FillRealize`` (a
``torch.autograd.Function``) puts a realization into a torch graph with
gradients for the data map and the band-power amplitudes of P(k).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = [
    "FillOpts", "FillStats", "FillError", "load", "lib_path", "fill_opts_default",
    "fill_init", "fill_realize", "fill_ml", "fill_relax", "fill_subdivide", "fill_set_annuli",
    "fill_laplace_ms", "fill_draw", "fill_apply", "fill_history",
    "fill_lanczos", "fill_time_pass", "fill_set_bands", "fill_backward", "fill_autotune", "fill_group_init",
    "fill_group_realize", "fill_group_size", "fill_group_destroy", "Group", "fill_apply_static",
    "fill_masked_count", "fill_destroy", "fill_strerror", "fill_last_error",
    "fill_version", "fill_realize_batch", "fill_set_spectrum", "Plan", "MODES",
    "EXPORTED_SYMBOLS", "BandPowerSpectrum", "FillRealize", "fill_realize_autograd",
    "realize_batch",
]

MODES = {"fp64": 0, "fp32": 1, "mixed": 2}
STATUS = {0: "FILL_OK", 1: "FILL_EINVAL", 2: "FILL_ENOMEM", 3: "FILL_ENOTCONV",
          4: "FILL_EBREAKDOWN", 5: "FILL_ETIMEOUT", 6: "FILL_ECUDA"}
EXPORTED_SYMBOLS = [
    "fill_opts_default", "fill_init", "fill_realize", "fill_ml", "fill_relax", "fill_subdivide",
    "fill_set_annuli", "fill_laplace_ms", "fill_draw", "fill_apply",
    "fill_history", "fill_lanczos", "fill_time_pass", "fill_set_bands", "fill_backward",
    "fill_autotune",
    "fill_group_init", "fill_group_realize", "fill_group_size", "fill_group_destroy",
    "fill_apply_static", "fill_masked_count", "fill_destroy", "fill_strerror",
    "fill_last_error", "fill_version", "fill_realize_batch", "fill_set_spectrum",
]


class FillOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("precond", ctypes.c_int),
                ("batch", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("host_loops", ctypes.c_int),
                ("inner_tol", ctypes.c_double),
                ("history_cap", ctypes.c_int), ("rows_per_cta", ctypes.c_int),
                ("ffts_per_cta", ctypes.c_int), ("backward", ctypes.c_int),
                ("update_delta", ctypes.c_double), ("col_kernel", ctypes.c_int),
                ("lanes", ctypes.c_int)]


class FillStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("status", ctypes.c_int), ("launches", ctypes.c_int),
                ("rel_resid", ctypes.c_double), ("true_rel_resid", ctypes.c_double),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class FillError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: {STATUS.get(status, status)} ({fill_strerror(status)})"
        if status == 6 or (status == 1 and where in ("fill_apply_static", "fill_subdivide",
                                                     "fill_set_spectrum")):
            msg += ": " + fill_last_error()
        super().__init__(msg)
        self.status = status


_LIB = None
_vp, _ci, _cd, _cll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong


def lib_path() -> str:
    return _build.lib_path()


def load() -> ctypes.CDLL:
    """Load ``libcgfill.so`` (built by ``__graft_entry__.build()``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = ctypes.CDLL(path)
    lib.fill_opts_default.argtypes = [ctypes.POINTER(FillOpts)]
    lib.fill_opts_default.restype = None
    lib.fill_init.argtypes = [ctypes.POINTER(_vp), _ci, _ci, _vp, _vp,
                              ctypes.POINTER(FillOpts), _vp]
    lib.fill_init.restype = _ci
    lib.fill_realize.argtypes = [_vp, _vp, _cll, _vp, _cd, _vp, ctypes.POINTER(FillStats)]
    lib.fill_realize.restype = _ci
    lib.fill_ml.argtypes = [_vp, _vp, _cll, _cd, _vp, ctypes.POINTER(FillStats)]
    lib.fill_ml.restype = _ci
    lib.fill_relax.argtypes = [_vp, _vp, _cll, _ci, _vp, ctypes.POINTER(FillStats)]
    lib.fill_relax.restype = _ci
    lib.fill_subdivide.argtypes = [_ci, _ci, _vp, _cd, _cd, _vp, _vp, _vp]
    lib.fill_subdivide.restype = _ci
    lib.fill_set_annuli.argtypes = [_vp, _ci, _vp, _vp]
    lib.fill_set_annuli.restype = _ci
    lib.fill_laplace_ms.argtypes = [_vp, _vp, _cll, _ci, _vp, _vp, ctypes.POINTER(FillStats)]
    lib.fill_laplace_ms.restype = _ci
    lib.fill_draw.argtypes = [_vp, _vp, _vp]
    lib.fill_draw.restype = _ci
    lib.fill_apply.argtypes = [_vp, _ci, _vp, _vp]
    lib.fill_apply.restype = _ci
    lib.fill_history.argtypes = [_vp, _ci, _vp, _ci, ctypes.POINTER(_ci)]
    lib.fill_history.restype = _ci
    lib.fill_lanczos.argtypes = [_vp, _ci, _vp, _vp, _ci, ctypes.POINTER(_ci),
                                 ctypes.POINTER(_cd), ctypes.POINTER(_cd)]
    lib.fill_lanczos.restype = _ci
    lib.fill_time_pass.argtypes = [_vp, _ci, _ci, _ci, ctypes.POINTER(_cd), ctypes.POINTER(_cd)]
    lib.fill_time_pass.restype = _ci
    lib.fill_set_bands.argtypes = [_vp, _ci, _vp, _vp]
    lib.fill_set_bands.restype = _ci
    lib.fill_backward.argtypes = [_vp, _vp, _cll, _vp, _cd, _vp, _vp, ctypes.POINTER(FillStats)]
    lib.fill_backward.restype = _ci
    lib.fill_autotune.argtypes = [_vp, ctypes.c_char_p]
    lib.fill_autotune.restype = _ci
    lib.fill_group_init.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ci, _ci,
                                    ctypes.c_char_p]
    lib.fill_group_init.restype = _ci
    lib.fill_group_realize.argtypes = [_vp, ctypes.POINTER(_vp), _vp, _cd, ctypes.POINTER(_vp),
                                       ctypes.POINTER(FillStats)]
    lib.fill_group_realize.restype = _ci
    lib.fill_group_size.argtypes = [_vp]
    lib.fill_group_size.restype = _ci
    lib.fill_group_destroy.argtypes = [_vp]
    lib.fill_group_destroy.restype = None
    lib.fill_apply_static.argtypes = [_ci, _ci, _vp, _vp, _ci, _vp, _vp, _vp]
    lib.fill_apply_static.restype = _ci
    lib.fill_realize_batch.argtypes = [ctypes.POINTER(_vp), _ci, ctypes.POINTER(_vp), _vp, _cd,
                                       ctypes.POINTER(_vp), ctypes.POINTER(FillStats)]
    lib.fill_realize_batch.restype = _ci
    lib.fill_set_spectrum.argtypes = [_vp, _vp]
    lib.fill_set_spectrum.restype = _ci
    lib.fill_masked_count.argtypes = [_vp]
    lib.fill_masked_count.restype = _cll
    lib.fill_destroy.argtypes = [_vp]
    lib.fill_destroy.restype = None
    lib.fill_strerror.argtypes = [_ci]
    lib.fill_strerror.restype = ctypes.c_char_p
    lib.fill_last_error.argtypes = []
    lib.fill_last_error.restype = ctypes.c_char_p
    lib.fill_version.argtypes = []
    lib.fill_version.restype = _ci
    _LIB = lib
    return lib


# ------------------------------------------------------------ C-ABI mirrors

def fill_opts_default() -> FillOpts:
    o = FillOpts()
    load().fill_opts_default(ctypes.byref(o))
    return o


def fill_init(ny, nx, P_half, observed, opts: FillOpts, stream: int = 0) -> int:
    P = np.ascontiguousarray(P_half, dtype=np.float64)
    m = np.ascontiguousarray(observed, dtype=np.uint8)
    if P.shape != (ny, nx // 2 + 1) or m.shape != (ny, nx):
        raise ValueError("P_half must be ny x (nx/2+1) and observed ny x nx")
    plan = _vp()
    st = load().fill_init(ctypes.byref(plan), int(ny), int(nx), P.ctypes.data, m.ctypes.data,
                          ctypes.byref(opts), _vp(stream))
    if st != 0:
        raise FillError(st, "fill_init")
    return plan.value


def fill_realize(plan, d_ptr, d_stride, seeds, tol, out_ptr, batch):
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    stats = (FillStats * batch)()
    st = load().fill_realize(_vp(plan), _vp(d_ptr), _cll(d_stride), s.ctypes.data,
                             _cd(tol), _vp(out_ptr), stats)
    return st, [x.as_dict() for x in stats]


def fill_ml(plan, d_ptr, d_stride, tol, out_ptr, batch):
    stats = (FillStats * batch)()
    st = load().fill_ml(_vp(plan), _vp(d_ptr), _cll(d_stride), _cd(tol), _vp(out_ptr), stats)
    return st, [x.as_dict() for x in stats]


def fill_relax(plan, d_ptr, d_stride, iters, out_ptr, batch):
    stats = (FillStats * batch)()
    st = load().fill_relax(_vp(plan), _vp(d_ptr), _cll(d_stride), int(iters), _vp(out_ptr),
                           stats)
    return st, [x.as_dict() for x in stats]


def fill_subdivide(observed, delta, threshold=0.03, stream=None):
    """Boundary layer of width ``delta`` (Sect. 6.2) of a device uint8 mask
    (1 = observed): returns a device uint8 map, 1 on the layer's pixels."""
    import torch
    if not (isinstance(observed, torch.Tensor) and observed.is_cuda and
            observed.dtype == torch.uint8 and observed.dim() == 2 and observed.is_contiguous()):
        raise ValueError("observed: expected a contiguous 2-D uint8 CUDA tensor")
    ny, nx = observed.shape
    scratch = torch.empty(ny * (nx + 1), dtype=torch.int32, device=observed.device)
    layer = torch.empty_like(observed)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = load().fill_subdivide(ny, nx, _vp(observed.data_ptr()), float(delta), float(threshold),
                               _vp(scratch.data_ptr()), _vp(layer.data_ptr()), _vp(s.cuda_stream))
    if st != 0:
        raise FillError(st, "fill_subdivide")
    return layer


def fill_set_annuli(plan, r_in, r_out):
    a = np.ascontiguousarray(r_in, dtype=np.float64)
    b = np.ascontiguousarray(r_out, dtype=np.float64)
    st = load().fill_set_annuli(_vp(plan), int(a.size), a.ctypes.data, b.ctypes.data)
    if st != 0:
        raise FillError(st, "fill_set_annuli")


def fill_laplace_ms(plan, d_ptr, d_stride, iters, cls_ptr, out_ptr, batch):
    stats = (FillStats * batch)()
    st = load().fill_laplace_ms(_vp(plan), _vp(d_ptr), _cll(d_stride), int(iters), _vp(cls_ptr),
                                _vp(out_ptr), stats)
    return st, [x.as_dict() for x in stats]


def fill_draw(plan, seeds, out_ptr):
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    st = load().fill_draw(_vp(plan), s.ctypes.data, _vp(out_ptr))
    if st != 0:
        raise FillError(st, "fill_draw")


def fill_apply(plan, which, in_ptr, out_ptr):
    st = load().fill_apply(_vp(plan), int(which), _vp(in_ptr), _vp(out_ptr))
    if st != 0:
        raise FillError(st, "fill_apply")


def fill_history(plan, inst, cap):
    buf = np.zeros(max(cap, 1), dtype=np.float64)
    cnt = _ci(0)
    st = load().fill_history(_vp(plan), int(inst), buf.ctypes.data, int(cap), ctypes.byref(cnt))
    if st != 0:
        raise FillError(st, "fill_history")
    return buf[: cnt.value].copy()


def fill_lanczos(plan, inst, cap):
    """CG coefficients and the Lanczos extreme eigenvalues of realization
    ``inst`` of the last realize: ``(alpha, beta, lmin, lmax)``."""
    a = np.zeros(max(cap, 1), dtype=np.float64)
    b = np.zeros(max(cap, 1), dtype=np.float64)
    cnt, lo, hi = _ci(0), _cd(0), _cd(0)
    st = load().fill_lanczos(_vp(plan), int(inst), a.ctypes.data, b.ctypes.data, int(cap),
                             ctypes.byref(cnt), ctypes.byref(lo), ctypes.byref(hi))
    if st != 0:
        raise FillError(st, "fill_lanczos")
    k = min(cnt.value, cap)
    return a[:k].copy(), b[:k].copy(), lo.value, hi.value


def fill_time_pass(plan, pass_id, precision, reps):
    ms, nbytes = _cd(0), _cd(0)
    st = load().fill_time_pass(_vp(plan), int(pass_id), int(precision), int(reps),
                               ctypes.byref(ms), ctypes.byref(nbytes))
    if st != 0:
        raise FillError(st, "fill_time_pass")
    return ms.value, nbytes.value


def fill_set_bands(plan, band_of_k, sig_half):
    b = np.ascontiguousarray(band_of_k, dtype=np.int32)
    sg = np.ascontiguousarray(sig_half, dtype=np.float64)
    st = load().fill_set_bands(_vp(plan), int(b.max()) + 1, b.ctypes.data, sg.ctypes.data)
    if st != 0:
        raise FillError(st, "fill_set_bands")
    return int(b.max()) + 1


def fill_backward(plan, d_ptr, d_stride, gx_ptr, tol, gd_ptr, nbands, batch):
    gb = np.zeros((batch, max(nbands, 1)), dtype=np.float64)
    stats = (FillStats * batch)()
    st = load().fill_backward(_vp(plan), _vp(d_ptr), _cll(d_stride), _vp(gx_ptr), _cd(tol),
                              _vp(gd_ptr), gb.ctypes.data if nbands else None, stats)
    return st, (gb if nbands else None), [x.as_dict() for x in stats]


def fill_autotune(plan, cache_path=None):
    st = load().fill_autotune(_vp(plan), cache_path.encode() if cache_path else None)
    if st != 0:
        raise FillError(st, "fill_autotune")


def fill_group_init(plans, autotune=False, cache_path=None):
    arr = (_vp * len(plans))(*plans)
    g = _vp()
    st = load().fill_group_init(ctypes.byref(g), arr, len(plans), 1 if autotune else 0,
                                cache_path.encode() if cache_path else None)
    if st != 0:
        raise FillError(st, "fill_group_init")
    return g.value


def fill_group_realize(group, d_ptrs, seeds, tol, out_ptrs, total):
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    d = (_vp * len(d_ptrs))(*d_ptrs)
    o = (_vp * len(out_ptrs))(*out_ptrs)
    stats = (FillStats * total)()
    st = load().fill_group_realize(_vp(group), d, s.ctypes.data, _cd(tol), o, stats)
    return st, [x.as_dict() for x in stats]


def fill_group_size(group) -> int:
    return int(load().fill_group_size(_vp(group)))


def fill_group_destroy(group) -> None:
    if group:
        load().fill_group_destroy(_vp(group))


def fill_apply_static(ny, nx, P_ptr, obs_ptr, which, in_ptr, out_ptr, stream=0):
    """Operator application without a plan or any allocation (device pointers)."""
    st = load().fill_apply_static(int(ny), int(nx), _vp(P_ptr), _vp(obs_ptr), int(which),
                                  _vp(in_ptr), _vp(out_ptr), _vp(stream))
    if st != 0:
        raise FillError(st, "fill_apply_static")


def fill_realize_batch(plans, d_ptrs, seeds, tol, out_ptrs, total):
    """Realizations for several plans in one call (one data map per plan)."""
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    pl = (_vp * len(plans))(*plans)
    d = (_vp * len(d_ptrs))(*d_ptrs)
    o = (_vp * len(out_ptrs))(*out_ptrs)
    stats = (FillStats * total)()
    st = load().fill_realize_batch(pl, len(plans), d, s.ctypes.data, _cd(tol), o, stats)
    return st, [x.as_dict() for x in stats]


def fill_set_spectrum(plan, P_half, ny, nx):
    P = np.ascontiguousarray(P_half, dtype=np.float64)
    if P.shape != (ny, nx // 2 + 1):
        raise ValueError("P_half must be ny x (nx/2+1)")
    st = load().fill_set_spectrum(_vp(plan), P.ctypes.data)
    if st != 0:
        raise FillError(st, "fill_set_spectrum")


def fill_masked_count(plan) -> int:
    return int(load().fill_masked_count(_vp(plan)))


def fill_destroy(plan) -> None:
    if plan:
        load().fill_destroy(_vp(plan))


def fill_strerror(status: int) -> str:
    return load().fill_strerror(int(status)).decode()


def fill_last_error() -> str:
    return load().fill_last_error().decode()


def fill_version() -> int:
    return int(load().fill_version())


# ------------------------------------------------------------ torch wrapper

class Plan:
    """A fill-in plan for one grid, spectrum and mask, fed with torch tensors.

    ``mode`` is ``"fp64"`` (plain FP64 PCG), ``"fp32"`` (FP32 operator,
    FP64-accurate inner products) or ``"mixed"`` (FP32 inner PCG with
    double-float residuals and reliable updates).  Maps are float32 in fp32
    mode and float64 otherwise, on the current CUDA device.  The remaining
    keywords mirror ``fill_opts`` (``lanes``: sub-batches of the CG loops run
    as parallel graph branches, 0 = automatic; ``rows_per_cta`` /
    ``ffts_per_cta``: the CG loop precision's CTA shapes, 0 = default).
    """

    def __init__(self, P_half, observed, mode="mixed", precond=True, batch=1,
                 max_iter=10000, max_refine=10, inner_tol=1e-6, history_cap=0,
                 rows_per_cta=0, ffts_per_cta=0, backward=False, update_delta=1e-2,
                 host_loops=False, col_kernel=0, lanes=0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1109_0286_gb300 needs a CUDA GPU; no CPU fallback exists")
        o = fill_opts_default()
        o.mode = MODES[mode]
        o.precond = 1 if precond else 0
        o.batch = int(batch)
        o.max_iter = int(max_iter)
        o.max_refine = int(max_refine)
        o.inner_tol = float(inner_tol)
        o.history_cap = int(history_cap)
        o.rows_per_cta = int(rows_per_cta)
        o.ffts_per_cta = int(ffts_per_cta)
        o.backward = 1 if backward else 0
        o.update_delta = float(update_delta)
        o.host_loops = 1 if host_loops else 0
        o.col_kernel = int(col_kernel)
        o.lanes = int(lanes)
        self.nbands = 0
        self.calls = 0          # compute calls so far (each may overwrite the device state)
        self.ny, self.nx = observed.shape
        self.batch = int(batch)
        self.mode = mode
        self.history_cap = int(history_cap)
        self.dtype = torch.float32 if mode == "fp32" else torch.float64
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self._plan = fill_init(self.ny, self.nx, P_half, observed, o, self._stream.cuda_stream)

    def _check(self, t, name, maps):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype
                and t.is_contiguous() and t.numel() == maps * self.ny * self.nx):
            raise ValueError(f"{name}: expected a contiguous {self.dtype} CUDA tensor "
                             f"with {maps} map(s) of {self.ny}x{self.nx}")

    def realize(self, d, seeds, tol, out=None, check=True):
        """Constrained realizations of data ``d`` (one map shared by the batch,
        or ``batch`` maps).  Returns ``(out, stats)``."""
        self.calls += 1
        import torch
        shared = d.numel() == self.ny * self.nx
        self._check(d, "d", 1 if shared else self.batch)
        if out is None:
            out = torch.empty((self.batch, self.ny, self.nx), dtype=self.dtype, device=d.device)
        self._check(out, "out", self.batch)
        seeds = np.asarray(seeds, dtype=np.uint64).reshape(-1)
        if seeds.size != self.batch:
            raise ValueError("need one seed per realization")
        st, stats = fill_realize(self._plan, d.data_ptr(), 0 if shared else self.ny * self.nx,
                                 seeds, tol, out.data_ptr(), self.batch)
        if check and st not in (0,):
            raise FillError(st, "fill_realize")
        return out, stats

    def ml(self, d, tol, out=None, check=True):
        """Maximum-likelihood fills x_M = -(Q_MM)^-1 Q_MU d_U of data ``d``
        (one map shared by the batch, or ``batch`` maps).  Returns
        ``(out, stats)``."""
        self.calls += 1
        import torch
        shared = d.numel() == self.ny * self.nx
        self._check(d, "d", 1 if shared else self.batch)
        if out is None:
            out = torch.empty((self.batch, self.ny, self.nx), dtype=self.dtype, device=d.device)
        self._check(out, "out", self.batch)
        st, stats = fill_ml(self._plan, d.data_ptr(), 0 if shared else self.ny * self.nx, tol,
                            out.data_ptr(), self.batch)
        if check and st != 0:
            raise FillError(st, "fill_ml")
        return out, stats

    def relax(self, d, iters, out=None, check=True):
        """Kernel-relaxation sweeps (Sect. 5, eq. Algo) from x_M = 0: returns
        ``(out, stats)``."""
        self.calls += 1
        import torch
        shared = d.numel() == self.ny * self.nx
        self._check(d, "d", 1 if shared else self.batch)
        if out is None:
            out = torch.empty((self.batch, self.ny, self.nx), dtype=self.dtype, device=d.device)
        self._check(out, "out", self.batch)
        st, stats = fill_relax(self._plan, d.data_ptr(), 0 if shared else self.ny * self.nx,
                               iters, out.data_ptr(), self.batch)
        if check and st != 0:
            raise FillError(st, "fill_relax")
        return out, stats

    def set_annuli(self, r_in, r_out):
        """Annuli of the kernel Laplace solver (Sect. 6.3)."""
        fill_set_annuli(self._plan, r_in, r_out)

    def laplace_ms(self, d, iters, cls, out=None, check=True):
        """Sweeps of the kernel Laplace solver with per-pixel annulus index
        ``cls`` (device uint8 map).  Returns ``(out, stats)``."""
        self.calls += 1
        import torch
        shared = d.numel() == self.ny * self.nx
        self._check(d, "d", 1 if shared else self.batch)
        if not (isinstance(cls, torch.Tensor) and cls.is_cuda and cls.dtype == torch.uint8
                and cls.numel() == self.ny * self.nx and cls.is_contiguous()):
            raise ValueError("cls: expected a contiguous uint8 CUDA map")
        if out is None:
            out = torch.empty((self.batch, self.ny, self.nx), dtype=self.dtype, device=d.device)
        self._check(out, "out", self.batch)
        st, stats = fill_laplace_ms(self._plan, d.data_ptr(), 0 if shared else self.ny * self.nx,
                                    iters, cls.data_ptr(), out.data_ptr(), self.batch)
        if check and st != 0:
            raise FillError(st, "fill_laplace_ms")
        return out, stats

    def set_spectrum(self, P_half):
        """Replace P(k) in place (``fill_set_spectrum``): new tables, no
        re-allocation; the mask, buffers and graphs are kept."""
        self.calls += 1
        fill_set_spectrum(self._plan, P_half, self.ny, self.nx)

    def set_bands(self, band_of_k, sig_half):
        """Band-power templates T_b(k) = 1[band(k) = b] S(k) for ``backward``."""
        self.nbands = fill_set_bands(self._plan, band_of_k, sig_half)

    def backward(self, d, grad_x, tol, grad_d=None, bands=True, check=True):
        """Adjoint gradients of L(x) through the last ``realize``: returns
        ``(dL/dd, dL/da_b or None, stats)``."""
        self.calls += 1
        import torch
        shared = d.numel() == self.ny * self.nx
        self._check(d, "d", 1 if shared else self.batch)
        self._check(grad_x, "grad_x", self.batch)
        if grad_d is None:
            grad_d = torch.empty((self.batch, self.ny, self.nx), dtype=self.dtype, device=d.device)
        self._check(grad_d, "grad_d", self.batch)
        nb = self.nbands if bands else 0
        st, gb, stats = fill_backward(self._plan, d.data_ptr(), 0 if shared else self.ny * self.nx,
                                      grad_x.data_ptr(), tol, grad_d.data_ptr(), nb, self.batch)
        if check and st != 0:
            raise FillError(st, "fill_backward")
        return grad_d, gb, stats

    def draw(self, seeds, out=None):
        self.calls += 1
        import torch
        if out is None:
            out = torch.empty((self.batch, self.ny, self.nx), dtype=self.dtype, device=self.device)
        self._check(out, "out", self.batch)
        fill_draw(self._plan, np.asarray(seeds, dtype=np.uint64).reshape(-1), out.data_ptr())
        return out

    def apply(self, which, x):
        """0: C^-1 x, 1: C^{1/2} x, 2: P_x C^-1 P_x x, 3: P_x C^{1/2} P_x x."""
        self.calls += 1
        import torch
        self._check(x, "x", 1)
        out = torch.empty_like(x)
        fill_apply(self._plan, which, x.data_ptr(), out.data_ptr())
        return out

    def time_pass(self, pass_id, precision=None, reps=20):
        """(ms per launch, algorithmic bytes per launch) of one hot-loop pass."""
        self.calls += 1
        if precision is None:
            precision = 1 if self.mode == "fp64" else 0
        return fill_time_pass(self._plan, pass_id, precision, reps)

    def autotune(self, cache_path=None):
        """Time the valid launch schedules (and, on mixed-radix grids, radix
        schedules) and keep the fastest."""
        self.calls += 1
        fill_autotune(self._plan, cache_path)

    def history(self, inst=0):
        return fill_history(self._plan, inst, self.history_cap)

    def lanczos(self, inst=0):
        """Lanczos estimate from the recorded CG coefficients (needs
        ``history_cap`` > 0): dict with alpha, beta, lmin, lmax, kappa."""
        a, b, lo, hi = fill_lanczos(self._plan, inst, self.history_cap)
        return {"alpha": a, "beta": b, "lmin": lo, "lmax": hi,
                "kappa": hi / lo if lo > 0 else float("inf")}

    @property
    def masked_count(self) -> int:
        return fill_masked_count(self._plan)

    def close(self):
        if getattr(self, "_plan", None):
            fill_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Many plans (masks, spectra, grid sizes) realized together: plans of one
    grid size share each pass launch, sizes run as concurrent graph branches."""

    def __init__(self, plans, autotune=False, cache_path=None):
        self.plans = list(plans)
        self._g = fill_group_init([p._plan for p in self.plans], autotune, cache_path)
        self.size = fill_group_size(self._g)

    def realize(self, ds, seeds, tol, outs=None, check=True):
        import torch
        if outs is None:
            outs = [torch.empty((p.batch, p.ny, p.nx), dtype=p.dtype, device=p.device)
                    for p in self.plans]
        for p, d, o in zip(self.plans, ds, outs):
            p._check(d, "d", 1)
            p._check(o, "out", p.batch)
        seeds = np.asarray(seeds, dtype=np.uint64).reshape(-1)
        if seeds.size != self.size:
            raise ValueError("need one seed per realization")
        st, stats = fill_group_realize(self._g, [d.data_ptr() for d in ds], seeds, tol,
                                       [o.data_ptr() for o in outs], self.size)
        if check and st != 0:
            raise FillError(st, "fill_group_realize")
        return outs, stats

    def close(self):
        if getattr(self, "_g", None):
            fill_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def realize_batch(plans, ds, seeds, tol, outs=None, check=True):
    """``fill_realize_batch``: realizations for several plans (masks, spectra
    and grid sizes may differ), one data map per plan.  Returns
    ``(outs, stats)`` with one output tensor of ``batch`` maps per plan."""
    import torch
    if outs is None:
        outs = [torch.empty((p.batch, p.ny, p.nx), dtype=p.dtype, device=p.device)
                for p in plans]
    for p, d, o in zip(plans, ds, outs):
        p._check(d, "d", 1)
        p._check(o, "out", p.batch)
        p.calls += 1
    total = sum(p.batch for p in plans)
    seeds = np.asarray(seeds, dtype=np.uint64).reshape(-1)
    if seeds.size != total:
        raise ValueError("need one seed per realization")
    st, stats = fill_realize_batch([p._plan for p in plans], [d.data_ptr() for d in ds], seeds,
                                   tol, [o.data_ptr() for o in outs], total)
    if check and st != 0:
        raise FillError(st, "fill_realize_batch")
    return outs, stats


# ------------------------------------------------------------ autograd

class BandPowerSpectrum:
    """Band-power parameterisation of the spectrum:
    ``P(k) = sum_b a_b 1[band(k) = b] S(k) + N(k)`` on the half plane
    ``ny x (nx/2+1)``; ``band_of_k`` (int), ``sig_half`` (S) and ``noise``
    (N, an array of that shape or a scalar) are host arrays.  The templates
    ``T_b = 1[band = b] S`` are what ``fill_set_bands`` receives, so the
    library's band gradient is dL/da_b."""

    def __init__(self, band_of_k, sig_half, noise):
        self.band_of_k = np.ascontiguousarray(band_of_k, dtype=np.int32)
        self.sig_half = np.ascontiguousarray(sig_half, dtype=np.float64)
        self.noise = noise
        self.nbands = int(self.band_of_k.max()) + 1

    def __call__(self, amps) -> np.ndarray:
        a = np.asarray(amps, dtype=np.float64).reshape(-1)
        if a.size != self.nbands:
            raise ValueError(f"need {self.nbands} band amplitudes")
        return a[self.band_of_k] * self.sig_half + self.noise


def _make_autograd():
    import torch

    class _FillRealize(torch.autograd.Function):
        """Constrained realizations as a differentiable torch operation.

        ``x = FillRealize.apply(d, amps, plan, model, seeds, tol)``: ``d`` is
        the data map (one map shared by the plan's batch, or ``batch`` maps),
        ``amps`` the band amplitudes a_b (host or device float64 tensor) of
        ``model`` (a ``BandPowerSpectrum``); the forward sets the plan's
        spectrum to ``model(amps)`` (``fill_set_spectrum``) when it differs
        from the current one and calls ``fill_realize``.  The backward calls
        ``fill_backward`` with the incoming dL/dx: one adjoint solve with the
        same operator and preconditioner gives dL/dd and dL/da_b (summed over
        the batch when ``d`` or ``amps`` are shared).  The draw's noise is held
        fixed by the seeds (a reparameterised gradient).  The plan needs
        ``backward=True``.  If the plan ran other work between the forward
        and the backward (another forward, a second backward), the backward
        first re-runs the same forward -- realizations are reproducible bit
        for bit from (d, P, seeds) -- so every backward sees its own
        realization.
        """

        @staticmethod
        def forward(ctx, d, amps, plan, model, seeds, tol):
            a = amps.detach().to("cpu", torch.float64).numpy().copy()
            _ensure_spectrum(plan, model, a)
            x, stats = plan.realize(d.detach(), seeds, tol)
            ctx.plan, ctx.model, ctx.seeds, ctx.tol, ctx.a = plan, model, seeds, tol, a
            ctx.amps_meta = (amps.device, amps.dtype, amps.shape)
            ctx.calls = plan.calls
            ctx.stats = stats
            ctx.save_for_backward(d)
            return x

        @staticmethod
        def backward(ctx, gx):
            (d,) = ctx.saved_tensors
            plan = ctx.plan
            if plan.calls != ctx.calls or not np.array_equal(plan._amps, ctx.a):
                _ensure_spectrum(plan, ctx.model, ctx.a)
                plan.realize(d.detach(), ctx.seeds, ctx.tol)
            want_bands = ctx.needs_input_grad[1]
            gx = gx.to(plan.dtype).contiguous()
            gd, gb, _ = plan.backward(d.detach(), gx, ctx.tol, bands=want_bands)
            grad_d = grad_a = None
            if ctx.needs_input_grad[0]:
                grad_d = gd.sum(0).reshape(d.shape) if d.numel() == plan.ny * plan.nx else \
                    gd.reshape(d.shape)
            if want_bands:
                dev, dt, shape = ctx.amps_meta
                grad_a = torch.from_numpy(gb.sum(0)).to(device=dev, dtype=dt).reshape(shape)
            return grad_d, grad_a, None, None, None, None

    return _FillRealize


def _ensure_spectrum(plan, model, a):
    """Give ``plan`` the spectrum ``model(a)`` and the band templates of
    ``model`` (only what changed)."""
    if getattr(plan, "_model", None) is not model:
        plan.set_bands(model.band_of_k, model.sig_half)
        plan._model = model
        plan._amps = None
    if getattr(plan, "_amps", None) is None or not np.array_equal(plan._amps, a):
        plan.set_spectrum(model(a))
        plan._amps = np.array(a, copy=True)


def fill_realize_autograd(d, amps, plan, model, seeds, tol):
    """Differentiable constrained realizations: ``FillRealize.apply``."""
    return FillRealize.apply(d, amps, plan, model, seeds, tol)


try:
    import torch as _torch
except ImportError:   # pragma: no cover
    _torch = None
FillRealize = _make_autograd() if _torch is not None else None
