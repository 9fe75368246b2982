"""Direct FP64 Cauchy sum (Sec. 2.5, Eq. fmm-E) on all host cores: the plain C
routine of cauchy_omp.c (OpenMP over rows), loaded with ctypes.

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  The tests pin it against
closed forms and the dense Cauchy matrix of gnk_dense; the benchmark times it
for the host's pair-evaluation rate.  The CUDA library never uses it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "cauchy_omp.c")
LIB = os.path.join(_HERE, "_build", "libcauchy_omp.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile cauchy_omp.c (gcc -O3 -fopenmp) unless the library is current."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC], check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_cauchy_sum.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int]
        _lib.oracle_cauchy_sum.restype = None
    return _lib


def cauchy_sum(et, w, threads: int | None = None) -> np.ndarray:
    """z_i = sum_{j != i} w_j / (eta_i - eta_j) for all i, on `threads` host
    threads (default: every core)."""
    et = np.ascontiguousarray(et, dtype=np.complex128)
    w = np.ascontiguousarray(w, dtype=np.complex128)
    if et.shape != w.shape or et.ndim != 1:
        raise ValueError("et and w must be 1-D arrays of equal length")
    z = np.empty_like(et)
    n = int(et.shape[0])
    _load().oracle_cauchy_sum(n, et.ctypes.data, w.ctypes.data, z.ctypes.data,
                              int(threads or os.cpu_count() or 1))
    return z
