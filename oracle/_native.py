"""Build and load the oracle's C transform (``oracle_fft.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The shared library is
compiled with the host C compiler into ``oracle/_lib/`` on first use, or by
``__graft_entry__.build()``, and rebuilt whenever the source changes (its
SHA-256 is stored beside the library).  Nothing here touches the CUDA path.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle_fft.c")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liboracle_fft.so")
STAMP = LIB + ".sha256"

_lib = None


def _digest() -> str:
    with open(SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def _current() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(STAMP)):
        return False
    with open(STAMP) as f:
        return f.read().strip() == _digest()


def build(force: bool = False) -> str:
    """Compile ``oracle_fft.c`` into ``_lib/liboracle_fft.so`` if needed."""
    if not force and _current():
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle's FFT")
    os.makedirs(LIBDIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=LIBDIR)
    os.close(fd)
    cmd = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", SRC, "-o", tmp, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        os.unlink(tmp)
        raise RuntimeError("building the oracle FFT failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)          # atomic: concurrent builders never see half a file
    fd, tmp = tempfile.mkstemp(dir=LIBDIR)
    with os.fdopen(fd, "w") as f:
        f.write(_digest())
    os.replace(tmp, STAMP)
    return LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        for name in ("oracle_fft2", "oracle_fft_rows"):
            fn = getattr(L, name)
            fn.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_void_p, ctypes.c_int,
                           ctypes.c_int]
            fn.restype = ctypes.c_int
        _lib = L
    return _lib
