"""Build the native library (libsdft.so) in-tree with nvcc for sm_103a.

Sources are compiled in parallel into `_build/`, then linked into
`paper_2211_15299_gb300/_lib/libsdft.so` with the CUDA runtime linked
statically. No CMake; a rebuild only recompiles sources whose inputs changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libsdft.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
# SDFT_BOUNDS_CHECK=1 in the environment builds the debug library with range
# checks in every kernel (see sdft_debug_bounds_violations in include/sdft.h).
if os.environ.get("SDFT_BOUNDS_CHECK", "0") not in ("", "0"):
    NVCC_FLAGS = NVCC_FLAGS + ["-DSDFT_BOUNDS_CHECK=1"]
SOURCES = ["plan.cpp", "autotune.cpp", "api.cu", "batch.cu", "level_f32.cu", "level_f32w3.cu", "level_f64.cu",
           "queue_f32.cu", "queue_f32w3.cu", "queue_f32st.cu", "queue_f32w3st.cu", "queue_f64.cu", "server.cu",
           "sas.cu", "inverse_f32.cu", "inverse_f64.cu", "level_df.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsdft")


def _digest(paths, extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for p in paths:
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _headers():
    out = [os.path.join(INCLUDE, f) for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h")]
    out += [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cuh", ".hpp", ".h"))]
    return out


def _compile(nvcc: str, src: str, obj: str, verbose: bool, xptxas: bool) -> None:
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc, *NVCC_FLAGS, "-x", "c++", "-c", src, "-o", obj]
    elif xptxas:
        cmd.insert(1, "-Xptxas=-v")
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 or (verbose and r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}")


def build(verbose: bool = False, force: bool = False, xptxas: bool = False) -> str:
    """Compile (if needed) and return the path of libsdft.so."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    headers = _headers()
    flags = " ".join(ARCH + NVCC_FLAGS)
    jobs = []
    objs = []
    for name in SOURCES:
        src = os.path.join(CSRC, name)
        tag = _digest([src] + headers, flags)
        obj = os.path.join(BUILD, f"{name}.{tag}.o")
        objs.append(obj)
        for old in os.listdir(BUILD):          # drop objects of older versions of this source
            if old.startswith(name + ".") and old.endswith(".o") and os.path.join(BUILD, old) != obj:
                os.remove(os.path.join(BUILD, old))
        if force or not os.path.exists(obj):
            jobs.append((src, obj))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda j: _compile(nvcc, j[0], j[1], verbose, xptxas), jobs))
    link_tag = _digest(objs, "link")
    stamp = LIB + ".stamp"
    if force or jobs or not os.path.exists(LIB) or not os.path.exists(stamp) or open(stamp).read() != link_tag:
        tmp = LIB + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "--cudart", "static", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of libsdft.so failed")
        os.replace(tmp, LIB)
        with open(stamp, "w") as fh:
            fh.write(link_tag)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(verbose=v, force="--force" in sys.argv, xptxas="--xptxas" in sys.argv))
