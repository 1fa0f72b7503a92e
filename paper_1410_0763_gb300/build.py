"""Build libart.so in-tree with nvcc for sm_103a (GB300).

Usage: ``python -m paper_1410_0763_gb300.build [--force]``.  The library is
written to ``paper_1410_0763_gb300/lib/libart.so`` (git-ignored).  Translation
units compile in parallel; no cmake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "lib")
LIB = os.path.join(OUT_DIR, "libart.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["art_api.cu", "art_wave.cu", "art_sweep_exact.cu", "art_geometry.cpp", "art_probe.cu", "art_noalloc.cu", "art_ion.cu",
           "art_net.cu", "art_ablation.cu"]
HEADERS = ["art_kernels.cuh", "art_wave.cuh", "art_geometry.hpp", "art_ctx.hpp", "art_net_kernels.cuh", "art_net_internal.hpp",
           "art_variants.inc"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libart")


def _defines() -> list[str]:
    """Preprocessor definitions chosen by the environment (checked, profiling and tuning builds)."""
    d = []
    if os.environ.get("ART_WAVE_CHECK") == "1":
        # the wavefront kernel tests every global index before it is used (slower; for checking runs)
        d.append("-DART_WAVE_CHECK")
    if os.environ.get("ART_WAVE_STATS") == "1":
        # the wavefront kernel counts its barrier and poll cycles (art_wave_counters; for profiling runs)
        d.append("-DART_WAVE_STATS")
    # extra definitions for tuning builds (e.g. "-DART_WAVE_PUB=8")
    d += [x for x in os.environ.get("ART_NVCC_DEFINES", "").split() if x.startswith("-D")]
    return d


def _stale() -> bool:
    """The library is missing, older than a source, or built with other definitions."""
    if not os.path.exists(LIB):
        return True
    try:
        with open(LIB + ".defines") as f:
            if f.read().split() != _defines():
                return True
    except OSError:
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, h) for h in ("art.h", "art_net.h")] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = nvcc_path()
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    defines = _defines()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH + defines
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src: str) -> str:
        obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-cudart", "static"] + ARCH + objs + ["-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(LIB + ".defines", "w") as f:
        f.write(" ".join(defines) + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
