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


C_USER = r"""
#include <stdio.h>
#include "pgc.h"
/* A C caller of every entry point family: compiled and linked, not run. */
int use_all(const int32_t* rp, const int32_t* ci, const int32_t* cp, const int32_t* ri,
            const int64_t* vo, const int64_t* no, int32_t* col) {
    int32_t rounds = 0, ncol = 0, rpg = 0, cpg = 0, maxr = 0;
    pgc_opts o;
    pgc_opts_init(&o);
    o.flags = PGC_NO_DEGREE_RULE | PGC_VALIDATE;
    pgc_status s = pgc_color_d1(4, rp, ci, 1u, col, &rounds, &ncol, &o, NULL);
    s = pgc_color_d2(4, rp, ci, 1u, col, &rounds, &ncol, NULL, NULL);
    s = pgc_color_pd2(3, 4, rp, ci, cp, ri, 1u, col, &rounds, &ncol, NULL, NULL);
    s = pgc_color_d1_batch(1, vo, no, rp, ci, 1u, col, &rpg, &cpg, &maxr, NULL, NULL);
    s = pgc_color_d1_noalloc(4, rp, ci, 1u, col, &rounds, &ncol, 0u, NULL);
    pgc_server* srv = NULL;
    int64_t id = 0;
    pgc_request_info info;
    if (pgc_server_create((size_t)1 << 30, 4, &srv) == PGC_OK) {
        int32_t done = 0;
        pgc_server_counters cnt;
        pgc_server_submit_d1(srv, 4, rp, ci, 1u, col, &id);
        pgc_server_poll(srv, id, &done, &info);
        pgc_server_submit_pd2(srv, 3, 4, rp, ci, cp, ri, 1u, col, &id);
        pgc_server_wait(srv, id, 1000, &info);
        pgc_server_stats(srv, &cnt);
        pgc_server_destroy(srv);
    }
    printf("%s %s %s\n", pgc_status_string(s), pgc_last_error(), pgc_version());
    return (int)pgc_release();
}
int main(void) { return 0; }
"""


@pytest.mark.parametrize("lang", ["c99", "c11", "c++17"])
def test_header_compiles_and_links_from_c(tmp_path, lang):
    """include/pgc.h is plain C (no torch or CUDA types): a C or C++ caller
    of every entry point compiles warning-free and links to libpgc.so."""
    import shutil
    import subprocess
    cc = "g++" if lang.startswith("c++") else "gcc"
    if shutil.which(cc) is None:
        pytest.skip(f"{cc} not available")
    lib = _native.build()
    src = tmp_path / ("user.cpp" if cc == "g++" else "user.c")
    src.write_text(C_USER)
    exe = tmp_path / "user"
    cmd = [cc, f"-std={lang}", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", HEADER_DIR,
           str(src), "-o", str(exe), "-L", os.path.dirname(lib), "-lpgc",
           f"-Wl,-rpath,{os.path.dirname(lib)}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("field,value,msg", [
    ("max_rounds", -1, b"max_rounds"), ("mid_degree", -5, b"degree"),
    ("hub_degree", -1, b"degree"), ("block", 96, b"block"), ("block", 2048, b"block"),
    ("block", 200, b"block"), ("grid_per_sm", -2, b"grid_per_sm"),
    ("timeout_ms", -1, b"timeout_ms")])
def test_invalid_options_rejected_without_gpu(field, value, msg):
    """Every entry point that takes pgc_opts checks it before any device
    work: an empty problem with a bad option is INVALID_ARG with a message
    naming the option, and with good options it is OK."""
    L = binding.lib()
    r, k = ctypes.c_int32(7), ctypes.c_int32(7)
    o = binding.PgcOptsC()
    L.pgc_opts_init(ctypes.byref(o))
    setattr(o, field, value)
    empty = (ctypes.c_int32 * 1)(0)
    calls = {
        "d1": lambda opts: L.pgc_color_d1(0, empty, None, 1, None, ctypes.byref(r),
                                          ctypes.byref(k), opts, None),
        "d2": lambda opts: L.pgc_color_d2(0, empty, None, 1, None, ctypes.byref(r),
                                          ctypes.byref(k), opts, None),
        "pd2": lambda opts: L.pgc_color_pd2(0, 0, empty, None, empty, None, 1, None,
                                            ctypes.byref(r), ctypes.byref(k), opts, None),
    }
    for name, call in calls.items():
        st = call(ctypes.byref(o))
        assert st == 1, (name, st)
        assert msg in L.pgc_last_error(), (name, L.pgc_last_error())
        good = binding.PgcOptsC()
        L.pgc_opts_init(ctypes.byref(good))
        good.block, good.mid_degree, good.hub_degree = 512, 32, 1024
        assert call(ctypes.byref(good)) == 0, name
        assert call(None) == 0 and r.value == 0 and k.value == 0, name
