"""Seeded synthetic inputs for the coloring library (graphs in int32 CSR).

This module makes inputs only; it holds none of the coloring method's
arithmetic and is shared by the tests, the benchmark and the oracle checks.
Large families are generated by ``gen.c`` (counter-based random stream,
OpenMP), small textbook graphs directly in numpy.

The families stand in for the paper's workloads (its Table 1 SuiteSparse
graphs and hexahedral meshes, its Table 2 Jacobian patterns, which are not
available here):

* ``stencil3d``    -- 3D 7-point / 27-point meshes (the paper's hexahedral
                       weak-scaling meshes are this family);
* ``rmat``         -- skewed-degree graphs (the social-network/kron rows);
* ``er``, ``grid2d`` -- the members of the batched workload;
* ``bipartite``    -- random Jacobian patterns for partial distance-2.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpgcgen.so")
_lock = threading.Lock()
_lib = None

# exp(-7), written out so that every host builds the same Poisson table
_EXP_MINUS = {7.0: 0.0009118819655545162}


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True,
                       stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True)   # serial build
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u64, p, d = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.c_void_p, ctypes.c_double)
            lib.gen_threads.restype = ctypes.c_int
            lib.gen_csr_from_edges.argtypes = [i32, i64, p, p, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, p, p, i64]
            lib.gen_csr_from_edges.restype = i64
            lib.gen_stencil3d_nnz.argtypes = [i32, i32, i32, ctypes.c_int]
            lib.gen_stencil3d_nnz.restype = i64
            lib.gen_stencil3d.argtypes = [i32, i32, i32, ctypes.c_int, p, p]
            lib.gen_stencil3d.restype = None
            lib.gen_grid2d_edges.argtypes = [i32, p, p]
            lib.gen_grid2d_edges.restype = i64
            lib.gen_rmat_edges.argtypes = [i32, i64, d, d, d, u64, ctypes.c_int, p, p]
            lib.gen_rmat_edges.restype = None
            lib.gen_er_edges.argtypes = [i32, i64, u64, p, p]
            lib.gen_er_edges.restype = None
            lib.gen_bipartite_lengths.argtypes = [i32, d, d, u64, p]
            lib.gen_bipartite_lengths.restype = i64
            lib.gen_bipartite_entries.argtypes = [i32, i32, u64, p, p, p, p]
            lib.gen_bipartite_entries.restype = None
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class CSR:
    """Symmetric (or, for bipartite row side, rectangular) int32 CSR."""
    row_ptr: np.ndarray
    col_idx: np.ndarray

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if len(self.row_ptr) else 0


@dataclass
class Bipartite:
    """Rows x columns pattern: CSR (rows -> columns) and CSC (columns -> rows)."""
    n_rows: int
    n_cols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    col_ptr: np.ndarray
    row_idx: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def csr_from_edges(n: int, src, dst, symmetrize=True, drop_loops=True, dedup=True) -> CSR:
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = len(src)
    cap = 2 * m if symmetrize else m
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(max(cap, 1), dtype=np.int32)
    nnz = lib.gen_csr_from_edges(n, m, _p(src), _p(dst), int(symmetrize), int(drop_loops),
                                 int(dedup), _p(row_ptr), _p(col), cap)
    if nnz < 0:
        raise RuntimeError("csr assembly failed")
    if nnz >= 2**31:
        raise ValueError("nnz does not fit int32")
    return CSR(row_ptr.astype(np.int32), col[:nnz].copy())


def stencil3d(nx: int, ny: int | None = None, nz: int | None = None, points: int = 7) -> CSR:
    """3D 7-point or 27-point stencil; id = x + nx*(y + ny*z); sorted rows."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    assert points in (7, 27)
    lib = _load()
    n = nx * ny * nz
    nnz = lib.gen_stencil3d_nnz(nx, ny, nz, points)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    col = np.empty(max(nnz, 1), dtype=np.int32)
    lib.gen_stencil3d(nx, ny, nz, points, _p(row_ptr), _p(col))
    return CSR(row_ptr, col[:nnz])


def grid2d(n: int) -> CSR:
    """2D 5-point grid over n vertices, w = ceil(sqrt(n)), last row partial."""
    lib = _load()
    src = np.empty(2 * n + 1, dtype=np.int32)
    dst = np.empty(2 * n + 1, dtype=np.int32)
    m = lib.gen_grid2d_edges(n, _p(src), _p(dst))
    return csr_from_edges(n, src[:m], dst[:m])


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, a=0.57, b=0.19, c=0.19,
         scramble: bool = True, n_vertices: int | None = None) -> CSR:
    """R-MAT, (2^scale) vertices, edge_factor * 2^scale samples, symmetrized,
    deduplicated, self-loops dropped.  With n_vertices < 2^scale, samples
    with an endpoint >= n_vertices are redrawn from the next counters."""
    lib = _load()
    nv = 1 << scale
    m = edge_factor * nv if n_vertices is None else edge_factor * n_vertices
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    lib.gen_rmat_edges(scale, m, a, b, c, seed, int(scramble), _p(src), _p(dst))
    if n_vertices is not None and n_vertices < nv:
        keep = (src < n_vertices) & (dst < n_vertices)
        src, dst = src[keep], dst[keep]
        extra_seed = seed
        while len(src) < m:
            extra_seed = (extra_seed * 6364136223846793005 + 1442695040888963407) % 2**64
            need = m - len(src)
            s2 = np.empty(2 * need, dtype=np.int32)
            d2 = np.empty(2 * need, dtype=np.int32)
            lib.gen_rmat_edges(scale, 2 * need, a, b, c, extra_seed, int(scramble), _p(s2), _p(d2))
            k = (s2 < n_vertices) & (d2 < n_vertices)
            src = np.concatenate([src, s2[k][:need]])
            dst = np.concatenate([dst, d2[k][:need]])
        nv = n_vertices
    return csr_from_edges(nv, src, dst)


def er(n: int, avg_degree: float, seed: int = 1) -> CSR:
    """Erdos-Renyi G(n, m) with m = round(n * avg_degree / 2) samples;
    repeats and loops removed (so slightly fewer edges)."""
    lib = _load()
    m = int(round(n * avg_degree / 2))
    src = np.empty(max(m, 1), dtype=np.int32)
    dst = np.empty(max(m, 1), dtype=np.int32)
    lib.gen_er_edges(n, m, seed, _p(src), _p(dst))
    return csr_from_edges(n, src[:m], dst[:m])


def bipartite(n_rows: int, n_cols: int, lam: float = 7.0, seed: int = 1) -> Bipartite:
    """Rows of length 1 + Poisson(lam), uniform column ids, repeats in a row
    removed; returns CSR and CSC of the same pattern."""
    lib = _load()
    p0 = _EXP_MINUS.get(float(lam), math.exp(-lam))
    length = np.empty(n_rows, dtype=np.int32)
    total = lib.gen_bipartite_lengths(n_rows, float(lam), p0, seed, _p(length))
    off = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(length, out=off[1:])
    src = np.empty(max(total, 1), dtype=np.int32)
    dst = np.empty(max(total, 1), dtype=np.int32)
    lib.gen_bipartite_entries(n_rows, n_cols, seed, _p(length), _p(off), _p(src), _p(dst))
    src, dst = src[:total], dst[:total]
    rows = csr_from_edges(n_rows, src, dst, symmetrize=False, drop_loops=False)
    # CSC from the deduplicated CSR
    r = np.repeat(np.arange(n_rows, dtype=np.int32), np.diff(rows.row_ptr))
    cols = csr_from_edges(n_cols, rows.col_idx, r, symmetrize=False, drop_loops=False)
    return Bipartite(n_rows, n_cols, rows.row_ptr, rows.col_idx, cols.row_ptr, cols.col_idx)


# ------------------------------------------------------------------------
# small textbook graphs (numpy only)
# ------------------------------------------------------------------------
def from_edge_list(n: int, edges) -> CSR:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    adj = [set() for _ in range(n)]
    for u, v in e:
        if u != v:
            adj[u].add(int(v))
            adj[v].add(int(u))
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(a) for a in adj])
    col = np.array([u for a in adj for u in sorted(a)], dtype=np.int32)
    return CSR(row_ptr, col)


def complete(n: int) -> CSR:
    return from_edge_list(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def complete_bipartite(m: int, n: int) -> CSR:
    """Vertices 0..m-1 on one side, m..m+n-1 on the other."""
    return from_edge_list(m + n, [(i, m + j) for i in range(m) for j in range(n)])


def star(leaves: int) -> CSR:
    return from_edge_list(leaves + 1, [(0, j) for j in range(1, leaves + 1)])


def path(n: int) -> CSR:
    return from_edge_list(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n: int) -> CSR:
    return from_edge_list(n, [(i, (i + 1) % n) for i in range(n)])


def empty(n: int) -> CSR:
    return CSR(np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32))


def mycielski(k: int) -> CSR:
    """Mycielski graph M_k (M_2 = K_2); chromatic number k."""
    n, edges = 2, [(0, 1)]
    for _ in range(k - 2):
        # vertices 0..n-1, copies n..2n-1, apex 2n
        new = list(edges)
        for u, v in edges:
            new.append((u, n + v))
            new.append((v, n + u))
        new += [(n + i, 2 * n) for i in range(n)]
        edges, n = new, 2 * n + 1
    return from_edge_list(n, edges)


def random_small(n: int, p: float, seed: int) -> CSR:
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return from_edge_list(n, zip(iu[0][keep], iu[1][keep]))


def random_bipartite_small(n_rows: int, n_cols: int, p: float, seed: int) -> Bipartite:
    rng = np.random.default_rng(seed)
    m = rng.random((n_rows, n_cols)) < p
    rows = [np.nonzero(m[r])[0] for r in range(n_rows)]
    cols = [np.nonzero(m[:, c])[0] for c in range(n_cols)]
    rp = np.zeros(n_rows + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(x) for x in rows])
    cp = np.zeros(n_cols + 1, dtype=np.int32)
    cp[1:] = np.cumsum([len(x) for x in cols])
    ci = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    ri = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return Bipartite(n_rows, n_cols, rp, ci, cp, ri)


# ------------------------------------------------------------------------
# the batched workload: many graphs of uneven size, flattened
# ------------------------------------------------------------------------
@dataclass
class Batch:
    """G graphs flattened: graph g's vertices are [vtx_off[g], vtx_off[g+1]),
    its local row_ptr (n_g + 1 entries, starting at 0) sits at
    row_ptr[vtx_off[g] + g : vtx_off[g+1] + g + 1] and its local column ids
    at col_idx[nnz_off[g] : nnz_off[g+1]]."""
    vtx_off: np.ndarray   # int64[G+1]
    nnz_off: np.ndarray   # int64[G+1]
    row_ptr: np.ndarray   # int32[N + G]
    col_idx: np.ndarray   # int32[NNZ]

    @property
    def num_graphs(self) -> int:
        return len(self.vtx_off) - 1

    def graph(self, g: int) -> CSR:
        a, b = int(self.vtx_off[g]), int(self.vtx_off[g + 1])
        rp = self.row_ptr[a + g: b + g + 1]
        e0, e1 = int(self.nnz_off[g]), int(self.nnz_off[g + 1])
        return CSR(rp.copy(), self.col_idx[e0:e1].copy())


def make_batch(graphs) -> Batch:
    G = len(graphs)
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    nnz_off = np.zeros(G + 1, dtype=np.int64)
    vtx_off[1:] = np.cumsum([g.n for g in graphs])
    nnz_off[1:] = np.cumsum([g.nnz for g in graphs])
    row_ptr = np.concatenate([g.row_ptr for g in graphs]).astype(np.int32) if G else \
        np.zeros(0, np.int32)
    col_idx = np.concatenate([g.col_idx for g in graphs]).astype(np.int32) if G else \
        np.zeros(0, np.int32)
    return Batch(vtx_off, nnz_off, row_ptr, col_idx)


def batch_plan(num_graphs: int = 4096, n_min: int = 100, n_max: int = 200_000, seed: int = 1):
    """Sizes (log-uniform on [n_min, n_max]) and ER average degrees (U[2, 32])
    of the mixed batch."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), num_graphs)).astype(np.int64)
    degs = rng.uniform(2.0, 32.0, num_graphs)
    return sizes, degs


def batch_member(i: int, sizes, degs, seed: int = 1) -> CSR:
    """Member i: a 2D 5-point grid for even i, G(n, m) for odd i."""
    n = int(sizes[i])
    if i % 2 == 0:
        return grid2d(n)
    return er(n, float(degs[i]), seed=seed * 1000003 + i)


def batch_mixed(num_graphs: int = 4096, n_min: int = 100, n_max: int = 200_000,
                seed: int = 1) -> Batch:
    """Even members: 2D 5-point grids; odd members: G(n, m) with average
    degree U[2, 32]; sizes log-uniform on [n_min, n_max]."""
    sizes, degs = batch_plan(num_graphs, n_min, n_max, seed)
    return make_batch([batch_member(i, sizes, degs, seed) for i in range(num_graphs)])
