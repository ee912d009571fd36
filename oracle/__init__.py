"""CPU oracle for the speculate-and-resolve coloring -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it, and nothing here imports the product.

The arithmetic lives in ``pgc_oracle.c`` (plain single-threaded C, built with
gcc into ``oracle/_build/liboracle.so``); this module only marshals numpy
arrays through ctypes.  ``setbased.py`` holds a second, independently written
pure-Python restatement used to cross-check the C code on tiny graphs.

Each entry point follows the paper (Bogle et al., arXiv 2107.00075):
D1 = Sec. 3.2 with Alg. 3/4, D2 = Sec. 3.5 with Alg. 5, PD2 = Sec. 3.6 with
Alg. 5 (doPartialColoring), the loser rule = Alg. 4 with recolorDegrees
(Sec. 3.3), first-fit = Alg. 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pgc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

D1, D2, PD2, PD2B = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile pgc_oracle.c with gcc (plain C11, -O2, no vector intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _declare(lib):
    if True:
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        p = ctypes.c_void_p
        lib.oracle_splitmix64.argtypes = [u64]
        lib.oracle_splitmix64.restype = u64
        lib.oracle_v_is_recolored.argtypes = [i32, u64, i32, i32, u64, i32, i32]
        lib.oracle_v_is_recolored.restype = ctypes.c_int
        sig = [i32, p, p, u64, i32, i32, p, p, p, p, p, i32]
        lib.oracle_color_d1.argtypes = sig
        lib.oracle_color_d1.restype = ctypes.c_int
        lib.oracle_color_d2.argtypes = sig
        lib.oracle_color_d2.restype = ctypes.c_int
        lib.oracle_color_pd2.argtypes = [i32, i32, p, p, p, p, u64, i32, i32,
                                         p, p, p, p, p, i32]
        lib.oracle_color_pd2.restype = ctypes.c_int
        lib.oracle_color_d1_priority.argtypes = sig
        lib.oracle_color_d1_priority.restype = ctypes.c_int
        lib.oracle_color_pd2_bipartite.argtypes = lib.oracle_color_pd2.argtypes
        lib.oracle_color_pd2_bipartite.restype = ctypes.c_int
        for name in ("oracle_count_improper", "oracle_count_non_grundy"):
            f = getattr(lib, name)
            f.argtypes = [i32, i32, i32, p, p, p, p, p]
            f.restype = i64
        return lib


def load_library(path: str):
    """Load a compiled copy of pgc_oracle.c (the default one, or a mutant a
    test compiled to show that the pins catch a planted mistake)."""
    return _declare(ctypes.CDLL(path))


def compile_source(src_text: str, out_path: str) -> str:
    """Compile C source text (e.g. a mutated copy of the oracle) to out_path."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", out_path, c_path], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


@dataclass
class Result:
    colors: np.ndarray
    rounds: int
    num_colors: int
    trace_w: np.ndarray   # |W_r| for r = 1..rounds
    trace_s: np.ndarray   # sum of deg(v) over W_r


def splitmix64(x: int, lib=None) -> int:
    return int(_load(lib).oracle_splitmix64(ctypes.c_uint64(x & (2**64 - 1))))


def v_is_recolored(deg_v, rand_v, v, deg_u, rand_u, u, recolor_degrees=True,
                   lib=None) -> bool:
    """Alg. 4's decision for a pair with equal colors: True if v is recolored."""
    return bool(_load(lib).oracle_v_is_recolored(deg_v, rand_v, v, deg_u, rand_u, u,
                                              int(recolor_degrees)))


_ERR = {-1: "invalid argument", -2: "out of memory", -3: "did not converge"}


def _finish(rc, colors, rounds, ncol, tw, ts):
    if rc != 0:
        raise RuntimeError(f"oracle failed: {_ERR.get(rc, rc)}")
    r = int(rounds.value)
    return Result(colors, r, int(ncol.value), tw[:r].copy(), ts[:r].copy())


def color_d1(row_ptr, col_idx, seed=1, recolor_degrees=True, max_rounds=0,
             trace_cap=100000, lib=None) -> Result:
    return _color(D1, row_ptr, col_idx, seed, recolor_degrees, max_rounds, trace_cap, lib)


PRIO_DYNAMIC, PRIO_SATURATION = 1, 2


def color_d1_priority(row_ptr, col_idx, mode, seed=1, max_rounds=0, trace_cap=100000,
                      lib=None) -> Result:
    """D1 whose Alg. 4 degree term is the dynamic degree (mode 1: uncolored
    adjacency entries) or the saturation degree (mode 2: distinct colors
    1..deg+1 among colored neighbors), taken at the start of each round
    (Sec. 3.3, closing paragraph)."""
    lib = _load(lib)
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = len(rp) - 1
    colors = np.zeros(max(n, 0), dtype=np.int32)
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    tw = np.zeros(trace_cap, dtype=np.int64)
    ts = np.zeros(trace_cap, dtype=np.int64)
    rc = lib.oracle_color_d1_priority(n, _ptr(rp), _ptr(ci), ctypes.c_uint64(seed), int(mode),
                                      max_rounds, _ptr(colors), ctypes.byref(rounds),
                                      ctypes.byref(ncol), _ptr(tw), _ptr(ts), trace_cap)
    return _finish(rc, colors, rounds, ncol, tw, ts)


def color_d2(row_ptr, col_idx, seed=1, recolor_degrees=True, max_rounds=0,
             trace_cap=100000, lib=None) -> Result:
    return _color(D2, row_ptr, col_idx, seed, recolor_degrees, max_rounds, trace_cap, lib)


def _color(kind, row_ptr, col_idx, seed, recolor_degrees, max_rounds, trace_cap, lib):
    lib = _load(lib)
    rp, ci = _i32(row_ptr), _i32(col_idx)
    n = len(rp) - 1
    colors = np.zeros(max(n, 0), dtype=np.int32)
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    tw = np.zeros(trace_cap, dtype=np.int64)
    ts = np.zeros(trace_cap, dtype=np.int64)
    f = lib.oracle_color_d1 if kind == D1 else lib.oracle_color_d2
    rc = f(n, _ptr(rp), _ptr(ci), ctypes.c_uint64(seed), int(recolor_degrees), max_rounds,
           _ptr(colors), ctypes.byref(rounds), ctypes.byref(ncol), _ptr(tw), _ptr(ts),
           trace_cap)
    return _finish(rc, colors, rounds, ncol, tw, ts)


def color_pd2(n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, seed=1,
              recolor_degrees=True, max_rounds=0, trace_cap=100000, lib=None) -> Result:
    lib = _load(lib)
    rp, ci, cp, ri = _i32(row_ptr), _i32(col_idx), _i32(col_ptr), _i32(row_idx)
    colors = np.zeros(n_cols, dtype=np.int32)
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    tw = np.zeros(trace_cap, dtype=np.int64)
    ts = np.zeros(trace_cap, dtype=np.int64)
    rc = lib.oracle_color_pd2(n_rows, n_cols, _ptr(rp), _ptr(ci), _ptr(cp), _ptr(ri),
                              ctypes.c_uint64(seed), int(recolor_degrees), max_rounds,
                              _ptr(colors), ctypes.byref(rounds), ctypes.byref(ncol),
                              _ptr(tw), _ptr(ts), trace_cap)
    return _finish(rc, colors, rounds, ncol, tw, ts)


def color_pd2_bipartite(n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, seed=1,
                        recolor_degrees=True, max_rounds=0, trace_cap=100000,
                        lib=None) -> Result:
    """PD2 over every vertex of the bipartite graph (Sec. 3.6): colors of the
    n_cols columns (ids 0..n_cols-1) then of the n_rows rows (ids n_cols + i);
    two vertices conflict when they share a neighbor."""
    lib = _load(lib)
    rp, ci, cp, ri = _i32(row_ptr), _i32(col_idx), _i32(col_ptr), _i32(row_idx)
    colors = np.zeros(n_cols + n_rows, dtype=np.int32)
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    tw = np.zeros(trace_cap, dtype=np.int64)
    ts = np.zeros(trace_cap, dtype=np.int64)
    rc = lib.oracle_color_pd2_bipartite(n_rows, n_cols, _ptr(rp), _ptr(ci), _ptr(cp), _ptr(ri),
                                        ctypes.c_uint64(seed), int(recolor_degrees), max_rounds,
                                        _ptr(colors), ctypes.byref(rounds), ctypes.byref(ncol),
                                        _ptr(tw), _ptr(ts), trace_cap)
    return _finish(rc, colors, rounds, ncol, tw, ts)


def _check(fname, kind, n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, colors):
    lib = _load()
    rp, ci = _i32(row_ptr), _i32(col_idx)
    cp = None if col_ptr is None else _i32(col_ptr)
    ri = None if row_idx is None else _i32(row_idx)
    c = _i32(colors)
    r = getattr(lib, fname)(kind, n_rows, n_cols, _ptr(rp), _ptr(ci), _ptr(cp), _ptr(ri),
                            _ptr(c))
    if r < 0:
        raise RuntimeError(f"{fname}: {_ERR.get(int(r), r)}")
    return int(r)


def count_improper(kind, row_ptr, col_idx, colors, n_rows=None, n_cols=None,
                   col_ptr=None, row_idx=None) -> int:
    """Equal-colored pairs within the problem's neighborhood (+ uncolored vertices)."""
    n = len(row_ptr) - 1
    return _check("oracle_count_improper", kind, n if n_rows is None else n_rows,
                  n if n_cols is None else n_cols, row_ptr, col_idx, col_ptr, row_idx, colors)


def count_non_grundy(kind, row_ptr, col_idx, colors, n_rows=None, n_cols=None,
                     col_ptr=None, row_idx=None) -> int:
    """Vertices whose color is not the mex of their neighborhood's colors."""
    n = len(row_ptr) - 1
    return _check("oracle_count_non_grundy", kind, n if n_rows is None else n_rows,
                  n if n_cols is None else n_cols, row_ptr, col_idx, col_ptr, row_idx, colors)
