"""Build and load the native library (libpgc.so) for sm_103a.

The library is compiled in-tree with nvcc (``-gencode
arch=compute_103a,code=sm_103a``) into ``paper_2107_00075_gb300/_build``.
Loading fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import glob
import os
import shutil
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(_HERE, "csrc")
BUILD = os.path.join(_HERE, "_build")
LIB = os.path.join(BUILD, "libpgc.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(
        os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel, then link libpgc.so."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        nvcc = _nvcc()
        flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                        "-I", INCLUDE, "-I", CSRC]
        if verbose:
            flags += ["-Xptxas", "-v"]

        def compile_one(src):
            obj = os.path.join(BUILD, os.path.basename(src) + ".o")
            cmd = [nvcc] + flags + ["-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            return obj, r.stderr

        with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            results = list(ex.map(compile_one, sources()))
        objs = [o for o, _ in results]
        if verbose:
            for _, log in results:
                print(log)
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcuda"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        return LIB


def load():
    """Load libpgc.so (building it first if sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(path)
    return _lib
