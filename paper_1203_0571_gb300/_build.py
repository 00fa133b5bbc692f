"""Build libfse.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel to an object file, then one
shared-library link.  The CUDA runtime is linked shared so that libfse and
PyTorch use the same runtime (and therefore the same device pointers and
streams).  Output: paper_1203_0571_gb300/_build/libfse.so (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfse.so")
SOURCES = ["fse_api.cu", "fse_kernels.cu", "fse_adjoint.cu", "fse_ragged.cu", "fse_star.cu", "fse_moment_grad.cu", "fse_cutout.cu"]
HEADERS = ["fse_internal.h", "fse_device.cuh", os.path.join(INCLUDE, "fse.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--cudart", "shared",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfse")
    return p


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


PEAKS_LIB = os.path.join(OUT_DIR, "libfse_peaks.so")
PEAKS_SOURCES = ["pipe_peaks.cu"]


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile (if needed) and return the path of libfse.so (libfse_peaks.so too)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    hdrs = [h if os.path.isabs(h) else os.path.join(CSRC, h) for h in HEADERS]
    hdrs.append(os.path.join(INCLUDE, "fse_peaks.h"))
    objs = []
    jobs = []
    for src in SOURCES + PEAKS_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc()] + ARCH + FLAGS + (extra or []) + ["-c", s, "-o", o]
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode:
                print(" ".join(cmd))
                print(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    n = len(SOURCES)
    for lib, lobjs in ((LIB, objs[:n]), (PEAKS_LIB, objs[n:])):
        if force or jobs or _stale(lib, lobjs):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nvcc()] + ARCH + ["-shared", "--cudart", "shared", "-o", tmp] + lobjs
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode:
                raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
