"""In-tree build of the CUDA library ``_lib/libcgfill.so`` for sm_103a.

Compiles the translation units in parallel with nvcc (one -gencode, static
cudart) and links them into one shared library with a plain C ABI.  Skips the
work only when a SHA-256 of every source, the header, this file and the
compiler flags, stored beside the library when it was built, matches the
current one (a copied or stale binary with newer timestamps is rebuilt).
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIBNAME = "libcgfill.so"
SOURCES = ["cg_launch_df_row0.cu", "cg_launch_df_row1.cu", "cg_launch_df_row2.cu",
           "cg_launch_f32_row0.cu", "cg_launch_f32_row1.cu", "cg_launch_f64_row0.cu",
           "cg_launch_f64_row1.cu", "cg_launch_df_col.cu", "cg_generic.cu", "cgfill.cu",
           "cg_launch_f32_col.cu", "cg_launch_f64_col.cu", "cg_launch_f32_row.cu",
           "cg_launch_f64_row.cu", "cg_launch_df_row.cu", "cg_static.cu", "cg_subdivide.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcgfill")


def source_digest() -> str:
    """SHA-256 over the sources, the header, this build script and the flags."""
    h = hashlib.sha256()
    deps = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC))
    deps += [os.path.join(ROOT, "include", "cgfill.h"), os.path.abspath(__file__)]
    for d in deps:
        if os.path.isfile(d):
            h.update(os.path.basename(d).encode())
            with open(d, "rb") as f:
                h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _stamp(target: str) -> str:
    return target + ".sha256"


def _stale(target: str) -> bool:
    if not (os.path.exists(target) and os.path.exists(_stamp(target))):
        return True
    with open(_stamp(target)) as f:
        return f.read().strip() != source_digest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library if needed; return its path."""
    target = lib_path()
    if not force and not _stale(target):
        return target
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    nvcc = _nvcc()
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(LIBDIR, "obj", src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    errors = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"--- {src}\n{out}")
        elif verbose and out.strip():
            print(out)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = target + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, target)
    with open(_stamp(target) + ".tmp", "w") as f:
        f.write(source_digest())
    os.replace(_stamp(target) + ".tmp", _stamp(target))
    return target


if __name__ == "__main__":
    print(build(force=True, verbose=True))
