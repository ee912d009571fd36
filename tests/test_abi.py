"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/pgc.h declares; host-side argument checks
that need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2107_00075_gb300 import _native, binding

HEADER_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared_functions():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pgc_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("pgc_color_d1", "pgc_last_error", "pgc_status_string", "pgc_release",
                 "pgc_opts_init", "pgc_version"):
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_native.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_status_strings_and_version():
    L = binding.lib()
    assert L.pgc_status_string(0) == b"PGC_OK"
    assert L.pgc_status_string(4) == b"PGC_ERR_NO_CONVERGE"
    assert b"sm_103a" in L.pgc_version()


def test_opts_struct_layout():
    # the ctypes mirror must match the C layout: 8 int32 fields then a pointer
    assert ctypes.sizeof(binding.PgcOptsC) == 8 * 4 + 8
    assert binding.PgcProfileC.kernel_ms.offset == 8 + 8 + 8 + 4 + 4


def test_host_argument_checks_without_gpu():
    """Argument errors are reported before any device work."""
    L = binding.lib()
    r, k = ctypes.c_int32(7), ctypes.c_int32(7)
    # n < 0
    st = L.pgc_color_d1(-1, None, None, 1, None, ctypes.byref(r), ctypes.byref(k), None, None)
    assert st == 1
    # NULL outputs
    st = L.pgc_color_d1(0, None, None, 1, None, None, None, None, None)
    assert st == 1
    # n == 0 is a valid empty problem
    st = L.pgc_color_d1(0, None, None, 1, None, ctypes.byref(r), ctypes.byref(k), None, None)
    assert st == 0 and r.value == 0 and k.value == 0
    # bad options
    o = binding.PgcOptsC()
    L.pgc_opts_init(ctypes.byref(o))
    o.block = 100
    st = L.pgc_color_d1(0, None, None, 1, None, ctypes.byref(r), ctypes.byref(k),
                        ctypes.byref(o), None)
    assert st == 1
    assert b"block" in L.pgc_last_error()
