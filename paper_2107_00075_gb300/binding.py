"""Thin Python binding of the C ABI in include/pgc.h (argument marshalling only).

Every computation runs in the CUDA library; these functions only turn torch
tensors / numpy arrays into pointers, call the C entry point of the same
name and raise on a non-OK status.  Arrays may live on the GPU (torch CUDA
tensors, used in place) or on the host (numpy arrays or CPU tensors, staged
by the library).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import _native

PGC_OK = 0
PGC_NO_DEGREE_RULE = 0x1
PGC_VALIDATE = 0x2
PGC_HOST_LOOP = 0x4
PGC_AUTOTUNE = 0x8
PGC_ASYNC = 0x10
PGC_PRIORITY_DYNAMIC = 0x20
PGC_PRIORITY_SATURATION = 0x40
PGC_MAX_KERNELS = 8

STATUS_NAMES = {0: "PGC_OK", 1: "PGC_ERR_INVALID_ARG", 2: "PGC_ERR_CUDA", 3: "PGC_ERR_OOM",
                4: "PGC_ERR_NO_CONVERGE", 5: "PGC_ERR_TIMEOUT", 6: "PGC_ERR_BUSY",
                7: "PGC_ERR_NOT_FOUND"}


class PgcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class PgcProfileC(ctypes.Structure):
    _fields_ = [("trace_w", ctypes.c_void_p), ("trace_s", ctypes.c_void_p),
                ("trace_h", ctypes.c_void_p), ("trace_cap", ctypes.c_int32), ("num_kernels", ctypes.c_int32),
                ("kernel_ms", ctypes.c_double * PGC_MAX_KERNELS),
                ("kernel_launches", ctypes.c_int64 * PGC_MAX_KERNELS),
                ("kernel_names", ctypes.c_char_p * PGC_MAX_KERNELS),
                ("launch_slot", ctypes.c_void_p), ("launch_ms", ctypes.c_void_p),
                ("launch_cap", ctypes.c_int32), ("num_launches", ctypes.c_int32),
                ("trace_nets", ctypes.c_void_p), ("trace_members", ctypes.c_void_p)]


class PgcOptsC(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("max_rounds", ctypes.c_int32),
                ("mid_degree", ctypes.c_int32), ("hub_degree", ctypes.c_int32),
                ("block", ctypes.c_int32), ("grid_per_sm", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int32), ("tail_vertices", ctypes.c_int32),
                ("profile", ctypes.POINTER(PgcProfileC))]


class RequestInfoC(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("num_colors", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("footprint_bytes", ctypes.c_int64)]


class ServerCountersC(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("active", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("bytes_in_use", ctypes.c_int64),
                ("peak_bytes", ctypes.c_int64), ("budget_bytes", ctypes.c_int64),
                ("max_active_seen", ctypes.c_int32), ("reserved", ctypes.c_int32)]


@dataclass
class Profile:
    """Per-round trace and (PGC_HOST_LOOP) per-kernel CUDA-event times."""
    trace_cap: int = 4096
    trace_w: np.ndarray = field(default=None)
    trace_s: np.ndarray = field(default=None)
    trace_h: np.ndarray = field(default=None)
    kernel_ms: dict = field(default_factory=dict)
    kernel_launches: dict = field(default_factory=dict)
    launch_cap: int = 0          # > 0: record every timed launch (host loop)
    launches: list = field(default_factory=list)   # [(kernel name, ms)]
    trace_nets: np.ndarray = field(default=None)     # D2/PD2: nets detection visited per round
    trace_members: np.ndarray = field(default=None)  # D2/PD2: their members per round


@dataclass
class ColorResult:
    colors: object
    rounds: int
    num_colors: int


_declared = False


def lib():
    """The loaded native library (raises if it cannot be built or loaded)."""
    global _declared
    L = _native.load()
    if not _declared:
        i32, u64, p = ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p
        L.pgc_color_d1.argtypes = [i32, p, p, u64, p, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(PgcOptsC), p]
        L.pgc_color_d1.restype = ctypes.c_int
        L.pgc_color_d2.argtypes = L.pgc_color_d1.argtypes
        L.pgc_color_d2.restype = ctypes.c_int
        L.pgc_color_pd2.argtypes = [i32, i32, p, p, p, p, u64, p, ctypes.POINTER(i32),
                                    ctypes.POINTER(i32), ctypes.POINTER(PgcOptsC), p]
        L.pgc_color_pd2.restype = ctypes.c_int
        L.pgc_color_pd2_bipartite.argtypes = L.pgc_color_pd2.argtypes
        L.pgc_color_pd2_bipartite.restype = ctypes.c_int
        L.pgc_color_d1_batch.argtypes = [i32, p, p, p, p, u64, p, p, p, ctypes.POINTER(i32),
                                         ctypes.POINTER(PgcOptsC), p]
        L.pgc_color_d1_batch.restype = ctypes.c_int
        L.pgc_color_d1_noalloc.argtypes = [i32, p, p, u64, p, ctypes.POINTER(i32),
                                           ctypes.POINTER(i32), ctypes.c_uint32, p]
        L.pgc_color_d1_noalloc.restype = ctypes.c_int
        L.pgc_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(p)]
        L.pgc_server_create.restype = ctypes.c_int
        L.pgc_server_submit_d1.argtypes = [p, i32, p, p, u64, p, ctypes.POINTER(ctypes.c_int64)]
        L.pgc_server_submit_d1.restype = ctypes.c_int
        L.pgc_server_submit_pd2.argtypes = [p, i32, i32, p, p, p, p, u64, p,
                                            ctypes.POINTER(ctypes.c_int64)]
        L.pgc_server_submit_pd2.restype = ctypes.c_int
        L.pgc_server_poll.argtypes = [p, ctypes.c_int64, ctypes.POINTER(i32),
                                      ctypes.POINTER(RequestInfoC)]
        L.pgc_server_poll.restype = ctypes.c_int
        L.pgc_server_wait.argtypes = [p, ctypes.c_int64, i32, ctypes.POINTER(RequestInfoC)]
        L.pgc_server_wait.restype = ctypes.c_int
        L.pgc_server_stats.argtypes = [p, ctypes.POINTER(ServerCountersC)]
        L.pgc_server_stats.restype = ctypes.c_int
        L.pgc_server_destroy.argtypes = [p]
        L.pgc_server_destroy.restype = ctypes.c_int
        L.pgc_last_error.restype = ctypes.c_char_p
        L.pgc_status_string.argtypes = [ctypes.c_int]
        L.pgc_status_string.restype = ctypes.c_char_p
        L.pgc_version.restype = ctypes.c_char_p
        L.pgc_release.restype = ctypes.c_int
        L.pgc_opts_init.argtypes = [ctypes.POINTER(PgcOptsC)]
        L.pgc_test_fail_alloc.argtypes = [i32]
        L.pgc_test_fail_alloc.restype = ctypes.c_int
        L.pgc_test_core_barrier.argtypes = [ctypes.c_uint32, i32, ctypes.c_uint32]
        L.pgc_test_core_barrier.restype = ctypes.c_int
        _declared = True
    return L


def _check(status: int):
    if status != PGC_OK:
        raise PgcError(status, lib().pgc_last_error().decode(errors="replace"))


class _Arr:
    """Pointer to an int32 array (torch tensor or numpy array), kept alive."""

    def __init__(self, a, name):
        self.obj = a
        self.device = None
        try:
            import torch
        except ImportError:  # pragma: no cover
            torch = None
        if torch is not None and isinstance(a, torch.Tensor):
            if a.dtype != torch.int32 or not a.is_contiguous():
                raise TypeError(f"{name} must be a contiguous int32 tensor")
            self.ptr = a.data_ptr()
            self.device = a.device if a.is_cuda else None
            self.n = a.numel()
        else:
            arr = np.asarray(a)
            if arr.dtype != np.int32 or not arr.flags.c_contiguous:
                raise TypeError(f"{name} must be a contiguous int32 array")
            self.obj = arr
            self.ptr = arr.ctypes.data
            self.n = arr.size


def _stream_handle(stream, device):
    import torch
    if stream is None:
        if device is None:
            return None
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _make_opts(flags, max_rounds, mid_degree, hub_degree, block, grid_per_sm, timeout_ms,
               profile: Optional[Profile], tail_vertices: int = 0):
    o = PgcOptsC()
    lib().pgc_opts_init(ctypes.byref(o))
    o.tail_vertices = tail_vertices
    o.flags, o.max_rounds = flags, max_rounds
    o.mid_degree, o.hub_degree = mid_degree, hub_degree
    o.block, o.grid_per_sm, o.timeout_ms = block, grid_per_sm, timeout_ms
    keep = []
    if profile is not None:
        pc = PgcProfileC()
        profile.trace_w = np.zeros(profile.trace_cap, dtype=np.int64)
        profile.trace_s = np.zeros(profile.trace_cap, dtype=np.int64)
        profile.trace_h = np.zeros(profile.trace_cap, dtype=np.int64)
        pc.trace_w = profile.trace_w.ctypes.data
        pc.trace_s = profile.trace_s.ctypes.data
        pc.trace_h = profile.trace_h.ctypes.data
        profile.trace_nets = np.zeros(profile.trace_cap, dtype=np.int64)
        profile.trace_members = np.zeros(profile.trace_cap, dtype=np.int64)
        pc.trace_nets = profile.trace_nets.ctypes.data
        pc.trace_members = profile.trace_members.ctypes.data
        pc.trace_cap = profile.trace_cap
        if profile.launch_cap > 0:
            profile._slots = np.zeros(profile.launch_cap, dtype=np.int32)
            profile._ms = np.zeros(profile.launch_cap, dtype=np.float32)
            pc.launch_slot = profile._slots.ctypes.data
            pc.launch_ms = profile._ms.ctypes.data
            pc.launch_cap = profile.launch_cap
        o.profile = ctypes.pointer(pc)
        keep.append(pc)
    return o, keep


def _finish_profile(profile: Optional[Profile], keep, rounds):
    if profile is None:
        return
    pc = keep[0]
    r = min(rounds, profile.trace_cap)
    profile.trace_w = profile.trace_w[:r].copy()
    profile.trace_s = profile.trace_s[:r].copy()
    profile.trace_h = profile.trace_h[:r].copy()
    profile.trace_nets = profile.trace_nets[:r].copy()
    profile.trace_members = profile.trace_members[:r].copy()
    for k in range(pc.num_kernels):
        name = pc.kernel_names[k]
        if name:
            profile.kernel_ms[name.decode()] = pc.kernel_ms[k]
            profile.kernel_launches[name.decode()] = pc.kernel_launches[k]
    if profile.launch_cap > 0:
        names = [(pc.kernel_names[k] or b"?").decode() for k in range(PGC_MAX_KERNELS)]
        m = min(pc.num_launches, profile.launch_cap)
        profile.launches = [(names[int(profile._slots[i])], float(profile._ms[i]))
                            for i in range(m)]


def _alloc_colors(n, device):
    if device is None:
        return np.zeros(n, dtype=np.int32)
    import torch
    return torch.empty(n, dtype=torch.int32, device=device)


def _device_ctx(device):
    import contextlib
    if device is None:
        return contextlib.nullcontext()
    import torch
    return torch.cuda.device(device)


def pgc_color_d1(row_ptr, col_idx, seed: int = 1, colors=None, *, flags: int = 0,
                 max_rounds: int = 0, mid_degree: int = 0, hub_degree: int = 0,
                 block: int = 0, grid_per_sm: int = 0, timeout_ms: int = 0,
                 tail_vertices: int = 0, profile: Optional[Profile] = None,
                 stream=None) -> ColorResult:
    """Distance-1 coloring of a symmetric int32 CSR graph (see pgc.h)."""
    return _color_sym("pgc_color_d1", row_ptr, col_idx, seed, colors, flags, max_rounds,
                      mid_degree, hub_degree, block, grid_per_sm, timeout_ms, profile, stream,
                      tail_vertices)


def pgc_color_d2(row_ptr, col_idx, seed: int = 1, colors=None, *, flags: int = 0,
                 max_rounds: int = 0, mid_degree: int = 0, hub_degree: int = 0,
                 block: int = 0, grid_per_sm: int = 0, timeout_ms: int = 0,
                 profile: Optional[Profile] = None, stream=None) -> ColorResult:
    """Distance-2 coloring of a symmetric int32 CSR graph (see pgc.h)."""
    return _color_sym("pgc_color_d2", row_ptr, col_idx, seed, colors, flags, max_rounds,
                      mid_degree, hub_degree, block, grid_per_sm, timeout_ms, profile, stream)


def pgc_color_pd2(n_rows: int, n_cols: int, row_ptr, col_idx, col_ptr, row_idx,
                  seed: int = 1, colors=None, *, flags: int = 0, max_rounds: int = 0,
                  block: int = 0, grid_per_sm: int = 0, timeout_ms: int = 0,
                  profile: Optional[Profile] = None, stream=None) -> ColorResult:
    """Partial distance-2 coloring of the columns of a pattern given as CSR
    and CSC (see pgc.h)."""
    rp, ci = _Arr(row_ptr, "row_ptr"), _Arr(col_idx, "col_idx")
    cp, ri = _Arr(col_ptr, "col_ptr"), _Arr(row_idx, "row_idx")
    if rp.n != n_rows + 1 or cp.n != n_cols + 1:
        raise ValueError("row_ptr/col_ptr sizes do not match n_rows/n_cols")
    if colors is None:
        colors = _alloc_colors(n_cols, rp.device)
    co = _Arr(colors, "colors")
    if co.n < n_cols:
        raise ValueError("colors is shorter than n_cols")
    o, keep = _make_opts(flags, max_rounds, 0, 0, block, grid_per_sm, timeout_ms, profile)
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    dev = rp.device or co.device
    with _device_ctx(dev):
        st = lib().pgc_color_pd2(n_rows, n_cols, rp.ptr, ci.ptr if ci.n else None, cp.ptr,
                                 ri.ptr if ri.n else None, ctypes.c_uint64(seed), co.ptr,
                                 ctypes.byref(rounds), ctypes.byref(ncol), ctypes.byref(o),
                                 _stream_handle(stream, dev))
    _check(st)
    _finish_profile(profile, keep, rounds.value)
    return ColorResult(colors, rounds.value, ncol.value)


def pgc_color_pd2_bipartite(n_rows: int, n_cols: int, row_ptr, col_idx, col_ptr, row_idx,
                            seed: int = 1, colors=None, *, flags: int = 0, max_rounds: int = 0,
                            block: int = 0, grid_per_sm: int = 0, timeout_ms: int = 0,
                            profile: Optional[Profile] = None, stream=None) -> ColorResult:
    """Partial distance-2 coloring of every vertex of the bipartite graph:
    colors[:n_cols] the columns, colors[n_cols + i] row i (see pgc.h)."""
    rp, ci = _Arr(row_ptr, "row_ptr"), _Arr(col_idx, "col_idx")
    cp, ri = _Arr(col_ptr, "col_ptr"), _Arr(row_idx, "row_idx")
    if rp.n != n_rows + 1 or cp.n != n_cols + 1:
        raise ValueError("row_ptr/col_ptr sizes do not match n_rows/n_cols")
    if colors is None:
        colors = _alloc_colors(n_cols + n_rows, rp.device)
    co = _Arr(colors, "colors")
    if co.n < n_cols + n_rows:
        raise ValueError("colors is shorter than n_cols + n_rows")
    o, keep = _make_opts(flags, max_rounds, 0, 0, block, grid_per_sm, timeout_ms, profile)
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    dev = rp.device or co.device
    with _device_ctx(dev):
        st = lib().pgc_color_pd2_bipartite(n_rows, n_cols, rp.ptr, ci.ptr if ci.n else None,
                                           cp.ptr, ri.ptr if ri.n else None,
                                           ctypes.c_uint64(seed), co.ptr, ctypes.byref(rounds),
                                           ctypes.byref(ncol), ctypes.byref(o),
                                           _stream_handle(stream, dev))
    _check(st)
    _finish_profile(profile, keep, rounds.value)
    return ColorResult(colors, rounds.value, ncol.value)


def _color_sym(fname, row_ptr, col_idx, seed, colors, flags, max_rounds, mid_degree,
               hub_degree, block, grid_per_sm, timeout_ms, profile, stream, tail_vertices=0):
    rp = _Arr(row_ptr, "row_ptr")
    ci = _Arr(col_idx, "col_idx")
    n = rp.n - 1
    if n < 0:
        raise ValueError("row_ptr must have n + 1 >= 1 entries")
    if colors is None:
        colors = _alloc_colors(n, rp.device)
    co = _Arr(colors, "colors")
    if co.n < n:
        raise ValueError("colors is shorter than n")
    o, keep = _make_opts(flags, max_rounds, mid_degree, hub_degree, block, grid_per_sm,
                         timeout_ms, profile, tail_vertices)
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    dev = rp.device or co.device
    with _device_ctx(dev):
        st = getattr(lib(), fname)(n, rp.ptr, ci.ptr if ci.n else None, ctypes.c_uint64(seed),
                                co.ptr, ctypes.byref(rounds), ctypes.byref(ncol),
                                ctypes.byref(o), _stream_handle(stream, dev))
    _check(st)
    _finish_profile(profile, keep, rounds.value)
    return ColorResult(colors, rounds.value, ncol.value)


def pgc_color_d1_noalloc(row_ptr, col_idx, seed: int = 1, colors=None, *, flags: int = 0,
                         stream=None) -> ColorResult:
    """Distance-1 coloring with no device allocation by the library (see
    pgc.h): CUDA tensors only, n <= 32768 and nnz <= 524288.  With colors
    None the output tensor is allocated here, by torch, before the call."""
    rp, ci = _Arr(row_ptr, "row_ptr"), _Arr(col_idx, "col_idx")
    n = rp.n - 1
    if n < 0:
        raise ValueError("row_ptr must have n + 1 >= 1 entries")
    if rp.device is None:
        raise TypeError("pgc_color_d1_noalloc takes CUDA tensors only")
    if colors is None:
        colors = _alloc_colors(n, rp.device)
    co = _Arr(colors, "colors")
    if co.n < n:
        raise ValueError("colors is shorter than n")
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    with _device_ctx(rp.device):
        st = lib().pgc_color_d1_noalloc(n, rp.ptr, ci.ptr if ci.n else None,
                                        ctypes.c_uint64(seed), co.ptr, ctypes.byref(rounds),
                                        ctypes.byref(ncol), flags,
                                        _stream_handle(stream, rp.device))
    _check(st)
    return ColorResult(colors, rounds.value, ncol.value)


@dataclass
class BatchResult:
    colors: object
    rounds_per_graph: object
    colors_per_graph: object
    rounds: int


class _Arr64:
    def __init__(self, a, name):
        try:
            import torch
        except ImportError:  # pragma: no cover
            torch = None
        self.device = None
        if torch is not None and isinstance(a, torch.Tensor):
            if a.dtype != torch.int64 or not a.is_contiguous():
                raise TypeError(f"{name} must be a contiguous int64 tensor")
            self.obj, self.ptr, self.n = a, a.data_ptr(), a.numel()
            self.device = a.device if a.is_cuda else None
        else:
            arr = np.ascontiguousarray(np.asarray(a, dtype=np.int64))
            self.obj, self.ptr, self.n = arr, arr.ctypes.data, arr.size


def pgc_color_d1_batch(vtx_off, nnz_off, row_ptr, col_idx, seed: int = 1, colors=None,
                       rounds_per_graph=None, colors_per_graph=None, *, flags: int = 0,
                       max_rounds: int = 0, mid_degree: int = 0, hub_degree: int = 0,
                       block: int = 0, grid_per_sm: int = 0, timeout_ms: int = 0,
                       tail_vertices: int = 0, profile: Optional[Profile] = None,
                       stream=None) -> BatchResult:
    """Batched distance-1 coloring of independent graphs (see pgc.h)."""
    vo, no = _Arr64(vtx_off, "vtx_off"), _Arr64(nnz_off, "nnz_off")
    rp, ci = _Arr(row_ptr, "row_ptr"), _Arr(col_idx, "col_idx")
    G = vo.n - 1
    if G < 0 or no.n != G + 1:
        raise ValueError("vtx_off and nnz_off must have G + 1 entries")
    N = rp.n - G
    dev = rp.device or vo.device
    if colors is None:
        colors = _alloc_colors(N, dev)
    if rounds_per_graph is None:
        rounds_per_graph = _alloc_colors(G, dev)
    if colors_per_graph is None:
        colors_per_graph = _alloc_colors(G, dev)
    co = _Arr(colors, "colors")
    gr, gc = _Arr(rounds_per_graph, "rounds_per_graph"), _Arr(colors_per_graph, "colors_per_graph")
    o, keep = _make_opts(flags, max_rounds, mid_degree, hub_degree, block, grid_per_sm,
                         timeout_ms, profile, tail_vertices)
    rounds = ctypes.c_int32(0)
    with _device_ctx(dev):
        st = lib().pgc_color_d1_batch(G, vo.ptr, no.ptr, rp.ptr, ci.ptr if ci.n else None,
                                      ctypes.c_uint64(seed), co.ptr, gr.ptr, gc.ptr,
                                      ctypes.byref(rounds), ctypes.byref(o),
                                      _stream_handle(stream, dev))
    _check(st)
    _finish_profile(profile, keep, rounds.value)
    return BatchResult(colors, rounds_per_graph, colors_per_graph, rounds.value)


def pgc_test_fail_alloc(after: int):
    """Test hook: the device allocation after `after` further successful ones
    fails once as out of memory (after < 0 disarms); see pgc.h."""
    _check(lib().pgc_test_fail_alloc(after))


def pgc_test_core_barrier(polls: int = 0, slow_block: int = -1, slow_us: int = 0):
    """Test hook: poll limit of the core loop's grid barrier (0: default) and
    a late core-loop block (-1: none); see pgc.h."""
    _check(lib().pgc_test_core_barrier(polls, slow_block, slow_us))


def pgc_release():
    _check(lib().pgc_release())


def pgc_version() -> str:
    return lib().pgc_version().decode()


@dataclass
class RequestInfo:
    status: int
    rounds: int
    num_colors: int
    t_submit_ns: int
    t_admit_ns: int
    t_done_ns: int
    footprint_bytes: int

    @property
    def latency_s(self) -> float:
        return (self.t_done_ns - self.t_submit_ns) * 1e-9


class PgcServer:
    """pgc_server_* (see pgc.h): continuous-batching coloring server.

    Keeps every submitted buffer alive until its request is reported done."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 16, device=None):
        import contextlib
        ctx = _device_ctx(device) if device is not None else contextlib.nullcontext()
        self._h = ctypes.c_void_p()
        with ctx:
            _check(lib().pgc_server_create(hbm_budget_bytes, max_active, ctypes.byref(self._h)))
        self._keep = {}

    def submit_d1(self, row_ptr, col_idx, seed: int = 1, colors=None) -> int:
        rp, ci = _Arr(row_ptr, "row_ptr"), _Arr(col_idx, "col_idx")
        n = rp.n - 1
        if colors is None:
            colors = np.zeros(n, dtype=np.int32)
        co = _Arr(colors, "colors")
        rid = ctypes.c_int64(0)
        _check(lib().pgc_server_submit_d1(self._h, n, rp.ptr, ci.ptr if ci.n else None,
                                          ctypes.c_uint64(seed), co.ptr, ctypes.byref(rid)))
        self._keep[rid.value] = (rp, ci, co)
        return rid.value

    def submit_pd2(self, n_rows, n_cols, row_ptr, col_idx, col_ptr, row_idx, seed: int = 1,
                   colors=None) -> int:
        arrs = [_Arr(a, nm) for a, nm in ((row_ptr, "row_ptr"), (col_idx, "col_idx"),
                                          (col_ptr, "col_ptr"), (row_idx, "row_idx"))]
        if colors is None:
            colors = np.zeros(n_cols, dtype=np.int32)
        co = _Arr(colors, "colors")
        rid = ctypes.c_int64(0)
        _check(lib().pgc_server_submit_pd2(self._h, n_rows, n_cols, arrs[0].ptr, arrs[1].ptr,
                                           arrs[2].ptr, arrs[3].ptr, ctypes.c_uint64(seed),
                                           co.ptr, ctypes.byref(rid)))
        self._keep[rid.value] = tuple(arrs) + (co,)
        return rid.value

    def colors(self, req_id: int):
        return self._keep[req_id][-1].obj

    def _info(self, ci) -> RequestInfo:
        return RequestInfo(ci.status, ci.rounds, ci.num_colors, ci.t_submit_ns, ci.t_admit_ns,
                           ci.t_done_ns, ci.footprint_bytes)

    def wait(self, req_id: int, timeout_ms: int = -1):
        """Returns (colors, RequestInfo) once done."""
        ci = RequestInfoC()
        _check(lib().pgc_server_wait(self._h, req_id, timeout_ms, ctypes.byref(ci)))
        keep = self._keep.pop(req_id)
        return keep[-1].obj, self._info(ci)

    def poll(self, req_id: int):
        """None while running, else (colors, RequestInfo)."""
        ci = RequestInfoC()
        done = ctypes.c_int32(0)
        st = lib().pgc_server_poll(self._h, req_id, ctypes.byref(done), ctypes.byref(ci))
        if not done.value:
            _check(st)
            return None
        keep = self._keep.pop(req_id)
        _check(st)
        return keep[-1].obj, self._info(ci)

    def stats(self) -> dict:
        c = ServerCountersC()
        _check(lib().pgc_server_stats(self._h, ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in ServerCountersC._fields_ if f != "reserved"}

    def close(self):
        if self._h:
            lib().pgc_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
