"""The batch autotuner's saved choices (csrc/tune_cache.h), host logic
compiled with g++: the file round-trips, lines that do not parse or hold a
configuration pgc_opts would reject are skipped (a damaged file must never
reach a launch), and the size classes group batches as documented."""
import ctypes
import math
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2107_00075_gb300", "csrc")

SHIM = r"""
#include "tune_cache.h"
#include <cstring>
using namespace pgc::d1;
extern "C" {
/* reads path, writes "key block mid hub;" for every entry into out */
int tc_read(const char* path, char* out, int cap) {
    std::FILE* fp = std::fopen(path, "r");
    if (!fp) return -1;
    std::map<std::string, Tuned> m;
    tune_file_read(fp, m);
    std::fclose(fp);
    std::string s;
    for (auto& kv : m)
        s += kv.first + " " + std::to_string(kv.second.block) + " " +
             std::to_string(kv.second.mid) + " " + std::to_string(kv.second.hub) + ";";
    if ((int)s.size() + 1 > cap) return -2;
    std::memcpy(out, s.c_str(), s.size() + 1);
    return (int)m.size();
}
int tc_append(const char* path, const char* key, int b, int mid, int hub) {
    std::FILE* fp = std::fopen(path, "a");
    if (!fp) return -1;
    tune_file_append(fp, key, Tuned{b, mid, hub});
    std::fclose(fp);
    return 0;
}
int tc_valid(int b, int mid, int hub) { return tuned_valid(Tuned{b, mid, hub}); }
void tc_class(long long n, long long nnz, int G, int use_deg, char* out) {
    std::strcpy(out, tune_size_class(n, nnz, G, use_deg != 0).c_str());
}
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("tune")
    src, so = d / "shim.cpp", d / "libtune.so"
    src.write_text(SHIM)
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-fPIC", "-shared",
                    "-I", CSRC, str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    L.tc_read.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int]
    L.tc_append.argtypes = [ctypes.c_char_p, ctypes.c_char_p] + [ctypes.c_int] * 3
    L.tc_valid.argtypes = [ctypes.c_int] * 3
    L.tc_class.argtypes = [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                           ctypes.c_char_p]
    return L


def _read(lib, path):
    buf = ctypes.create_string_buffer(1 << 16)
    k = lib.tc_read(str(path).encode(), buf, len(buf))
    assert k >= 0
    entries = [e.split() for e in buf.value.decode().split(";") if e]
    return {e[0]: tuple(int(x) for x in e[1:]) for e in entries}


def test_round_trip_and_later_lines_win(lib, tmp_path):
    f = tmp_path / "tune.txt"
    lib.tc_append(str(f).encode(), b"d1b:n26:d3:g12:r1", 256, 64, 16384)
    lib.tc_append(str(f).encode(), b"d1b:n20:d4:g1:r0", 512, 32, 1024)
    lib.tc_append(str(f).encode(), b"d1b:n26:d3:g12:r1", 128, 16, 256)
    assert _read(lib, f) == {"d1b:n26:d3:g12:r1": (128, 16, 256),
                             "d1b:n20:d4:g1:r0": (512, 32, 1024)}


def test_damaged_lines_are_skipped(lib, tmp_path):
    f = tmp_path / "tune.txt"
    f.write_text("good1 256 64 16384\n"
                 "garbage\n"
                 "zero_block 0 64 16384\n"
                 "odd_block 200 64 16384\n"
                 "huge_block 2048 64 16384\n"
                 "bad_tiers 256 64 32\n"
                 "no_mid 256 0 32\n"
                 "trailing 256 64 16384 7\n"
                 "short 256 64\n"
                 "good2 1024 128 16384\n")
    assert _read(lib, f) == {"good1": (256, 64, 16384), "good2": (1024, 128, 16384)}


def test_validity_matches_opts_limits(lib):
    for b in range(0, 1100, 8):
        assert lib.tc_valid(b, 16, 256) == (128 <= b <= 1024 and b % 32 == 0)
    assert lib.tc_valid(256, 64, 64) and not lib.tc_valid(256, 65, 64)
    assert not lib.tc_valid(256, 0, 64)


def test_size_classes(lib):
    out = ctypes.create_string_buffer(96)

    def cls(n, nnz, G, rd=True):
        lib.tc_class(n, nnz, G, int(rd), out)
        return out.value.decode()

    lg = lambda x: 0 if x <= 1 else int(round(math.log2(x)))
    # the 4096-graph workload: 108,006,486 vertices, 1,138,474,936 entries
    n, nnz = 108_006_486, 1_138_474_936
    assert cls(n, nnz, 4096) == f"d1b:n{lg(n)}:d{lg(nnz / n)}:g12:r1" == "d1b:n27:d3:g12:r1"
    assert cls(n, nnz, 4096, rd=False).endswith(":r0")
    assert cls(0, 0, 0) == "d1b:n0:d0:g0:r1"
    # batches whose sizes round to the same powers of two share a class
    assert cls(1000, 16000, 64) == cls(1100, 17000, 60)
    assert cls(1000, 16000, 64) != cls(4000, 64000, 64)
