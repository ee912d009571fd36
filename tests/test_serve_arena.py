"""The served form's HBM arena (csrc/arena.h), host logic compiled with g++
and checked against a brute-force model: first fit returns the lowest
offset with room, live ranges never overlap, the byte count in use is
exact, and freed neighbours coalesce (so an emptied arena is one range
again and can take a request of the whole budget)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2107_00075_gb300", "csrc")

SHIM = r"""
#include "arena.h"
using pgc::serve::Arena;
extern "C" {
void* arena_new(size_t cap) { Arena* a = new Arena(); a->init(cap); return a; }
int arena_alloc(void* a, size_t bytes, size_t* off) { return ((Arena*)a)->alloc(bytes, off); }
void arena_release(void* a, size_t off, size_t bytes) { ((Arena*)a)->release(off, bytes); }
size_t arena_used(void* a) { return ((Arena*)a)->used(); }
size_t arena_ranges(void* a) { return ((Arena*)a)->free_ranges(); }
void arena_delete(void* a) { delete (Arena*)a; }
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("arena")
    src, so = d / "shim.cpp", d / "libarena.so"
    src.write_text(SHIM)
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-fPIC", "-shared",
                    "-I", CSRC, str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    sz = ctypes.c_size_t
    L.arena_new.argtypes, L.arena_new.restype = [sz], ctypes.c_void_p
    L.arena_alloc.argtypes, L.arena_alloc.restype = [ctypes.c_void_p, sz,
                                                     ctypes.POINTER(sz)], ctypes.c_int
    L.arena_release.argtypes = [ctypes.c_void_p, sz, sz]
    L.arena_used.argtypes, L.arena_used.restype = [ctypes.c_void_p], sz
    L.arena_ranges.argtypes, L.arena_ranges.restype = [ctypes.c_void_p], sz
    L.arena_delete.argtypes = [ctypes.c_void_p]
    return L


def _first_fit(busy, bytes_):
    """Lowest offset of `bytes_` consecutive free units in the model."""
    free = ~busy
    run = 0
    for i, f in enumerate(free):
        run = run + 1 if f else 0
        if run == bytes_:
            return i - bytes_ + 1
    return None


@pytest.mark.parametrize("seed", range(6))
def test_arena_matches_first_fit_model(lib, seed):
    cap = 4096
    rng = np.random.default_rng(seed)
    a = lib.arena_new(cap)
    busy = np.zeros(cap, dtype=bool)
    live = {}
    off = ctypes.c_size_t(0)
    try:
        for step in range(1500):
            if live and (rng.random() < 0.45 or step % 97 == 0):
                k = list(live)[int(rng.integers(len(live)))]
                size = live.pop(k)
                lib.arena_release(a, k, size)
                busy[k:k + size] = False
            else:
                size = int(rng.integers(1, 400))
                want = _first_fit(busy, size)
                ok = lib.arena_alloc(a, size, ctypes.byref(off))
                assert bool(ok) == (want is not None)
                if ok:
                    assert off.value == want
                    assert not busy[want:want + size].any()
                    busy[want:want + size] = True
                    live[want] = size
            assert lib.arena_used(a) == int(busy.sum())
            # free ranges are maximal: one per run of free units
            runs = int(np.count_nonzero(np.diff(np.concatenate([[0], (~busy).astype(np.int8)])) == 1))
            assert lib.arena_ranges(a) == runs
        for k, size in list(live.items()):
            lib.arena_release(a, k, size)
        assert lib.arena_used(a) == 0 and lib.arena_ranges(a) == 1
        assert lib.arena_alloc(a, cap, ctypes.byref(off)) and off.value == 0
        assert not lib.arena_alloc(a, 1, ctypes.byref(off))
    finally:
        lib.arena_delete(a)


def test_arena_edge_cases(lib):
    off = ctypes.c_size_t(0)
    a = lib.arena_new(0)              # no budget: nothing fits
    assert not lib.arena_alloc(a, 1, ctypes.byref(off))
    lib.arena_delete(a)
    a = lib.arena_new(1000)
    assert not lib.arena_alloc(a, 1001, ctypes.byref(off))
    assert lib.arena_alloc(a, 1000, ctypes.byref(off)) and off.value == 0
    lib.arena_release(a, 0, 1000)
    # three blocks, free the middle then the outer ones: coalesces to one range
    offs = []
    for _ in range(3):
        assert lib.arena_alloc(a, 300, ctypes.byref(off))
        offs.append(off.value)
    assert offs == [0, 300, 600]
    lib.arena_release(a, 300, 300)
    assert lib.arena_ranges(a) == 2           # [300, 600) and [900, 1000)
    assert lib.arena_alloc(a, 100, ctypes.byref(off)) and off.value == 300   # first fit
    lib.arena_release(a, 300, 100)
    lib.arena_release(a, 0, 300)
    lib.arena_release(a, 600, 300)
    assert lib.arena_ranges(a) == 1 and lib.arena_used(a) == 0
    lib.arena_delete(a)
