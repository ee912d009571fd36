"""Multi-core CPU baseline -- BENCHMARK INFRASTRUCTURE, not the oracle.

``pgc_cpu_omp.c`` runs the oracle's distance-1 round loop on all host cores
with OpenMP (gcc ``-fopenmp``).  Its colors equal the oracle's bit for bit
(the tests check this); ``bench.py`` reports its rate beside the
single-core oracle.  It is compiled on first use, not by ``build()``, so a
host without OpenMP loses only this figure.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgc_cpu_omp.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libcpu_omp.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-Wall",
                    "-Wextra", "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, p = ctypes.c_int32, ctypes.c_void_p
            lib.cpu_omp_color_d1.argtypes = [i32, p, p, ctypes.c_uint64, i32, i32, i32, p,
                                             ctypes.POINTER(i32), ctypes.POINTER(i32),
                                             ctypes.POINTER(i32)]
            lib.cpu_omp_color_d1.restype = ctypes.c_int
            _lib = lib
        return _lib


def color_d1(row_ptr, col_idx, seed=1, recolor_degrees=True, threads=0):
    """Distance-1 coloring on `threads` cores (0: OpenMP's default).
    Returns (colors, rounds, num_colors, threads_used)."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    n = len(rp) - 1
    colors = np.zeros(max(n, 0), dtype=np.int32)
    rounds, ncol, used = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib.cpu_omp_color_d1(n, rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                              ctypes.c_uint64(seed), int(recolor_degrees), 0, int(threads),
                              colors.ctypes.data if n > 0 else None, ctypes.byref(rounds),
                              ctypes.byref(ncol), ctypes.byref(used))
    if rc != 0:
        raise RuntimeError(f"cpu_omp_color_d1 failed ({rc})")
    return colors, int(rounds.value), int(ncol.value), int(used.value)
