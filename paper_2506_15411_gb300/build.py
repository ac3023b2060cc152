"""Build libcbs.so (the CUDA library behind include/cbs.h) in-tree for sm_103a.

    python -m paper_2506_15411_gb300.build

Translation units are compiled in parallel with nvcc and linked into
paper_2506_15411_gb300/lib/libcbs.so.  A unit is rebuilt when it or a header is newer
than its object file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
OBJDIR = os.path.join(LIBDIR, "_build")
LIB = os.path.join(LIBDIR, "libcbs.so")

SOURCES = ["api.cu", "xpass.cu", "yzpass.cu", "ypass_tx4.cu", "ypass_tx8.cu", "ypass_tx16.cu", "zpass_tx4.cu",
           "zpass_tx8.cu", "zpass_tx16.cu", "misc.cu", "noalloc.cu", "design.cu", "serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs.append(os.path.join(ROOT, "include", "cbs.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, extra_flags=(), libdir: str = LIBDIR) -> str:
    """Compile (if stale) and link into libdir/libcbs.so; returns the library path.
    extra_flags (e.g. -D settings of the launch heuristics) are for builds kept apart in
    their own libdir."""
    objdir = os.path.join(libdir, "_build")
    lib = os.path.join(libdir, "libcbs.so")
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()
    hdr = _headers_mtime()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(objdir, src.replace(".cu", ".o"))
        if not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            jobs.append([cc, *ARCH, *FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, flush=True)

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(objdir, s.replace(".cu", ".o")) for s in SOURCES]
    if jobs or not os.path.exists(lib):
        tmp = lib + ".tmp"
        run([cc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
