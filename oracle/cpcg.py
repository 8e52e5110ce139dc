"""Loader of the oracle's C Jacobi-PCG (oracle/pcg_omp.c), the timed CPU baseline.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  ``build()`` compiles the C file with gcc and
OpenMP into ``oracle/_build/libpcg_omp.so``; ``jacobi_pcg`` runs it on a SciPy CSR matrix.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pcg_omp.c")
LIB = os.path.join(HERE, "_build", "libpcg_omp.so")
_lib = None


def build() -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the oracle's CPU baseline")
    cmd = [cc, "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("oracle C build failed:\n" + res.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp = C.c_void_p
        lib.oracle_jacobi_pcg.argtypes = [C.c_int64, vp, vp, vp, vp, vp, C.c_double, C.c_int64, vp, vp, vp, vp,
                                          C.POINTER(C.c_double)]
        lib.oracle_jacobi_pcg.restype = C.c_int64
        lib.oracle_threads.restype = C.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().oracle_threads())


def jacobi_pcg(A, f, u0=None, rtol=1e-8, max_iter=1_000_000):
    """(u, iterations, recurrence relative residual, seconds) of the C Jacobi-PCG on CSR A."""
    lib = _load()
    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    ptr = np.ascontiguousarray(A.indptr, np.int64)
    col = np.ascontiguousarray(A.indices, np.int32)
    val = np.ascontiguousarray(A.data, np.float64)
    f = np.ascontiguousarray(f, np.float64)
    u = np.zeros(n) if u0 is None else np.array(u0, np.float64)
    work = [np.empty(n) for _ in range(4)]
    rel = C.c_double()
    ptrs = [a.ctypes.data for a in (ptr, col, val, f, u)]
    t0 = time.perf_counter()
    it = lib.oracle_jacobi_pcg(n, *ptrs, rtol, max_iter, *[w.ctypes.data for w in work], C.byref(rel))
    sec = time.perf_counter() - t0
    return u, int(it), rel.value, sec
