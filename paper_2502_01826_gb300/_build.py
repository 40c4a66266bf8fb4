"""Compile libgsrf.so for sm_103a with nvcc (one -gencode, sources in parallel), and
libgsrf_peaks.so, the pipe-throughput microbenchmarks that give the render's roofline
its compute peaks."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
SO = os.path.join(PKG, "libgsrf.so")
PEAKS_SO = os.path.join(PKG, "libgsrf_peaks.so")
PEAKS_SRC = "peaks.cu"
SOURCES = ["gsrf_api.cu", "k_project.cu", "k_bin.cu", "k_dsort.cu", "k_render.cu", "k_signal.cu", "k_backward.cu", "gsrf_static.cu",
           "gsrf_tune.cu"]
HEADERS = ["gsrf_internal.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgsrf.so")


def _deps():
    out = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    out.append(os.path.join(ROOT, "include", "gsrf.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(SO) or not os.path.exists(PEAKS_SO):
        return False
    t = min(os.path.getmtime(SO), os.path.getmtime(PEAKS_SO))
    return all(os.path.getmtime(d) <= t for d in _deps() + [os.path.join(CSRC, PEAKS_SRC)])


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return SO
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = list(extra or [])

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-I", os.path.join(ROOT, "include"), "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        objs = list(ex.map(compile_one, SOURCES + [PEAKS_SRC]))
    for target, parts in ((SO, objs[:-1]), (PEAKS_SO, objs[-1:])):
        tmp = target + ".tmp%d" % os.getpid()
        r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *parts], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, target)
    return SO


if __name__ == "__main__":
    import sys
    print(build(force="-f" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "-v" in sys.argv else None))
