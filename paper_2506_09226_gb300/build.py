"""Build libqe.so (the CUDA operator library) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by its own nvcc process (in
parallel), then linked into paper_2506_09226_gb300/libqe.so.  The same units
are also compiled with -DQE_CHECKED into libqe_checked.so, the bounds-checked
build whose kernels test their write indices and report QE_ERR_DEVICE_CHECK
instead of writing out of bounds.  Objects go to
paper_2506_09226_gb300/_build/ (and _build/checked/).  A unit is rebuilt when
it or any header it may include is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libqe.so")
LIB_CHECKED = os.path.join(PKG, "libqe_checked.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(obj: str, src: str, hdr_mtime: float) -> bool:
    if not os.path.exists(obj):
        return True
    m = os.path.getmtime(obj)
    return m < os.path.getmtime(src) or m < hdr_mtime


def build(verbose: bool = False, extra_flags: list | None = None, checked: bool = True) -> str:
    """Compile and link libqe.so, and (checked=True) libqe_checked.so; the
    units of both are compiled in one pool.  Returns the path of libqe.so."""
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_mtime = max([os.path.getmtime(h) for h in _headers()] + [0.0])
    nvcc = _nvcc()
    variants = [(BUILD, LIB, NVCC_FLAGS + (extra_flags or []))]
    if checked:
        variants.append((os.path.join(BUILD, "checked"), LIB_CHECKED, NVCC_FLAGS + ["-DQE_CHECKED"] + (extra_flags or [])))
    jobs = []
    for bdir, _, flags in variants:
        os.makedirs(bdir, exist_ok=True)
        for src in srcs:
            obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
            if _stale(obj, src, hdr_mtime):
                jobs.append((src, obj, flags))

    def compile_one(job):
        src, obj, flags = job
        cmd = [nvcc] + flags + ["-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(compile_one, jobs):
            if verbose and out:
                sys.stderr.write(out)
    for bdir, lib, _ in variants:
        objs = [os.path.join(bdir, os.path.basename(s)[:-3] + ".o") for s in srcs]
        if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
            tmp = lib + f".tmp{os.getpid()}"
            r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stderr}")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
