"""Build libamh.so (the C-ABI library) and libamh_peaks.so (the roofline
microbenchmarks) in-tree for sm_103a with nvcc.

Each .cu file is compiled to an object in parallel, then linked into
``paper_2211_03193_gb300/libamh.so`` (or ``libamh_peaks.so``).  Objects go to
``_build/`` (ignored by git).  Rebuilds only when a source or header is newer
than the libraries.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libamh.so")
PEAKS_LIB = os.path.join(PKG, "libamh_peaks.so")

SOURCES = ["amh_api.cu", "amh_global.cu", "amh_gwarp.cu", "amh_local.cu", "amh_misc.cu",
           "amh_noalloc.cu"]
PEAKS_SOURCES = ["peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the AMH CUDA library cannot be built")


def _deps() -> list[str]:
    out = [os.path.join(CSRC, s) for s in SOURCES + PEAKS_SOURCES]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    out.append(os.path.abspath(__file__))
    return out


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(PEAKS_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAKS_LIB))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src: str) -> tuple[str, str]:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-I", CSRC, "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with ThreadPoolExecutor(len(SOURCES) + len(PEAKS_SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES + PEAKS_SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    objs = [o for o, _ in results]
    for lib, n0, n1 in ((LIB, 0, len(SOURCES)), (PEAKS_LIB, len(SOURCES), len(objs))):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs[n0:n1], "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        for _, log in results:
            f.write(log)
    return LIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True)
