"""Inputs and oracle runs for the full-size parity tests (run in spawned
worker processes: no CUDA here)."""
import oracle
from paper_2107_00075_gb300 import inputs as gen

import hashlib
import time

import numpy as np

CASES = ("rmat24_d1", "stencil128_d2", "bip_pd2")
BATCH_GRAPHS = 4096


def digest(colors) -> str:
    return hashlib.sha256(np.ascontiguousarray(colors, dtype=np.int32).tobytes()).hexdigest()


def batch_oracle_job(indices):
    """Oracle on members of the 4096-graph batch: (index, digest, rounds, colors)."""
    sizes, degs = gen.batch_plan(BATCH_GRAPHS)
    out = []
    for i in indices:
        g = gen.batch_member(i, sizes, degs)
        r = oracle.color_d1(g.row_ptr, g.col_idx, seed=1)
        out.append((i, digest(r.colors), r.rounds, r.num_colors))
    return out


def make_input(kind):
    if kind == "rmat24_d1":
        return gen.rmat(24, 16, seed=1)
    if kind == "stencil128_d2":
        return gen.stencil3d(128, 128, 128, points=27)
    if kind == "bip_pd2":
        return gen.bipartite(1 << 22, 1 << 20, lam=7.0, seed=1)
    raise ValueError(kind)


def oracle_job(kind):
    """The oracle on a full-size input: (colors, rounds, num_colors, trace_w,
    trace_s, {seconds, units}) -- the wall time of the coloring alone, the
    input generated before the clock starts; units = edges (D1, D2: nnz / 2)
    or entries (PD2: nnz)."""
    x = make_input(kind)
    t0 = time.perf_counter()
    if kind == "rmat24_d1":
        r = oracle.color_d1(x.row_ptr, x.col_idx, seed=1)
    elif kind == "stencil128_d2":
        r = oracle.color_d2(x.row_ptr, x.col_idx, seed=1)
    else:
        r = oracle.color_pd2(x.n_rows, x.n_cols, x.row_ptr, x.col_idx, x.col_ptr, x.row_idx,
                             seed=1)
    secs = time.perf_counter() - t0
    units = x.nnz if kind == "bip_pd2" else x.nnz / 2
    return r.colors, r.rounds, r.num_colors, r.trace_w, r.trace_s, {"seconds": secs,
                                                                      "units": units}
