"""ctypes access to oracle/alg1.c, the plain C restatement of Algorithm 1.

TEST INFRASTRUCTURE ONLY (part of the oracle): the tests and the bench's CPU
baseline / reference arm call it. `build()` compiles it with gcc (OpenMP when
available) into oracle/_lib; `alg1_batch` builds on first use if needed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alg1.c")
_LIB = os.path.join(_HERE, "_lib", "liboracle_alg1.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile alg1.c into a shared library (rebuilt when the source is newer)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)      # no OpenMP: one thread
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_alg1_batch.restype = ctypes.c_int
        _lib.oracle_alg1_batch.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
    return _lib


def alg1_batch(M: int, r, Jc, F, threads: int = 0):
    """Coefficients (N/k) F(J, I_r) f for every row of F (B, k) complex128, with
    Jc the canonical support and r the pivots; returns (C, threads used)."""
    lib = _load()
    r = np.ascontiguousarray(np.asarray(r, dtype=np.uint32))
    Jc = np.ascontiguousarray(np.asarray(Jc, dtype=np.uint64))
    F = np.ascontiguousarray(np.asarray(F, dtype=np.complex128))
    squeeze = F.ndim == 1
    if squeeze:
        F = F[None, :]
    C = np.empty_like(F)
    used = lib.oracle_alg1_batch(int(M), int(r.size), r.ctypes.data, Jc.ctypes.data, F.ctypes.data, C.ctypes.data,
                                 int(F.shape[0]), int(threads))
    if used < 0:
        raise ValueError("oracle_alg1_batch rejected its arguments")
    return (C[0] if squeeze else C), used
