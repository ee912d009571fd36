"""GPU parity for distance-2 and partial distance-2 coloring: the net-based
CUDA path through the C ABI must match the oracle (which walks two-hop
neighborhoods directly) bit for bit, with the per-round worklist trace."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2107_00075_gb300 import inputs as gen
from tests import _graphs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pgc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2107_00075_gb300 as p
    return p


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def d2_parity(pgc, g, seed=1, recolor_degrees=True, **kw):
    flags = kw.pop("flags", 0) | (0 if recolor_degrees else pgc.PGC_NO_DEGREE_RULE)
    prof = pgc.Profile(trace_cap=100000)
    r = pgc.pgc_color_d2(dev(g.row_ptr), dev(g.col_idx), seed=seed, flags=flags, profile=prof,
                         **kw)
    want = oracle.color_d2(g.row_ptr, g.col_idx, seed=seed, recolor_degrees=recolor_degrees)
    got = r.colors.cpu().numpy()
    assert r.rounds == want.rounds and r.num_colors == want.num_colors
    assert np.array_equal(got, want.colors), f"{np.count_nonzero(got != want.colors)} differ"
    assert np.array_equal(prof.trace_w, want.trace_w)
    assert np.array_equal(prof.trace_s, want.trace_s)
    return got


def pd2_parity(pgc, b, seed=1, recolor_degrees=True, **kw):
    flags = kw.pop("flags", 0) | (0 if recolor_degrees else pgc.PGC_NO_DEGREE_RULE)
    prof = pgc.Profile(trace_cap=100000)
    r = pgc.pgc_color_pd2(b.n_rows, b.n_cols, dev(b.row_ptr), dev(b.col_idx), dev(b.col_ptr),
                          dev(b.row_idx), seed=seed, flags=flags, profile=prof, **kw)
    want = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                            seed=seed, recolor_degrees=recolor_degrees)
    got = r.colors.cpu().numpy()
    assert r.rounds == want.rounds and r.num_colors == want.num_colors
    assert np.array_equal(got, want.colors), f"{np.count_nonzero(got != want.colors)} differ"
    assert np.array_equal(prof.trace_w, want.trace_w)
    assert np.array_equal(prof.trace_s, want.trace_s)
    return got


def test_worked_examples(pgc):
    cases = json.load(open(os.path.join(GOLDEN, "worked_examples.json")))["cases"]
    for c in cases:
        flags = 0 if c["recolor_degrees"] else pgc.PGC_NO_DEGREE_RULE
        if c["kind"] == "d2":
            g = gen.from_edge_list(c["n"], c["edges"])
            r = pgc.pgc_color_d2(dev(g.row_ptr), dev(g.col_idx), seed=c["seed"], flags=flags)
        elif c["kind"] == "pd2":
            b = _graphs.bipartite_from_rows(c["rows"], c["n_cols"])
            r = pgc.pgc_color_pd2(b.n_rows, b.n_cols, dev(b.row_ptr), dev(b.col_idx),
                                  dev(b.col_ptr), dev(b.row_idx), seed=c["seed"], flags=flags)
        else:
            continue
        assert list(r.colors.cpu().numpy()) == c["colors"] and r.rounds == c["rounds"], c["name"]


def test_d2_small_random(pgc):
    for i in range(40):
        g = gen.random_small(4 + i, 0.03 + (i % 6) * 0.06, seed=300 + i)
        d2_parity(pgc, g, seed=i + 1, recolor_degrees=bool(i % 3))


def test_d2_stencils(pgc):
    d2_parity(pgc, gen.stencil3d(12, 11, 10, points=27), seed=1)
    d2_parity(pgc, gen.stencil3d(20, 20, 20, points=7), seed=3)


def test_d2_large_nets(pgc):
    """Hubs give nets of more than 32 members (the chunked net path)."""
    g = gen.rmat(11, 8, seed=2)
    assert np.diff(g.row_ptr).max() > 32
    d2_parity(pgc, g, seed=4)


def test_pd2_random(pgc):
    for i in range(30):
        b = gen.random_bipartite_small(5 + i, 4 + 2 * i, 0.05 + (i % 5) * 0.08, seed=600 + i)
        pd2_parity(pgc, b, seed=i + 2, recolor_degrees=bool(i % 2))
    pd2_parity(pgc, gen.bipartite(40000, 10000, seed=5), seed=1)


def test_pd2_wide_rows(pgc):
    """Rows longer than 32 columns (large nets) and long columns (warp tier)."""
    b = gen.bipartite(3000, 200, lam=40.0, seed=7)
    assert np.diff(b.row_ptr).max() > 32 and np.diff(b.col_ptr).max() > 32
    pd2_parity(pgc, b, seed=9)


def _splitmix64(x):
    """splitmix64 (Steele, Lea, Flood 2014) on a uint64 array."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def test_pd2_equal_32bit_keys(pgc):
    """A hub column in all 2^17 rows makes the largest degree 18 bits wide.
    Detection first compares a 32-bit key (the degree, then the top hash bits
    that fit, the lowest of them cleared), so here only 13 hash bits count and
    columns of equal degree in one row often share it; the full key must then
    decide, as in the oracle."""
    R, k = 1 << 17, 7
    half = R * k // 2
    slots = np.arange(R * k, dtype=np.int64).reshape(R, k)
    other = 1 + slots % half                      # every other column in exactly 2 rows
    rows = np.concatenate([np.zeros((R, 1), np.int64), other], axis=1)
    n_cols = 1 + half
    row_ptr = np.arange(0, R * (k + 1) + 1, k + 1, dtype=np.int32)
    col_idx = rows.reshape(-1).astype(np.int32)
    entry_row = np.repeat(np.arange(R, dtype=np.int32), k + 1)
    order = np.argsort(col_idx, kind="stable")
    col_ptr = np.zeros(n_cols + 1, np.int32)
    col_ptr[1:] = np.cumsum(np.bincount(col_idx, minlength=n_cols))
    b = gen.Bipartite(R, n_cols, row_ptr, col_idx, col_ptr, entry_row[order])
    seed = 3
    # the instance holds many rows with two columns sharing that 32-bit key
    hi = _splitmix64(np.uint64(seed) ^ other.astype(np.uint64)) >> np.uint64(32)
    top = (~hi & np.uint64(0xFFFFFFFF)) >> np.uint64(18)
    top.sort(axis=1)
    assert np.count_nonzero((top[:, 1:] == top[:, :-1]).any(axis=1)) > 50
    pd2_parity(pgc, b, seed=seed)


def test_d2_equals_pd2_on_closed_neighborhoods(pgc):
    g = gen.random_small(60, 0.08, seed=17)
    b = _graphs.closed_neighborhood_matrix(g)
    a = pgc.pgc_color_d2(dev(g.row_ptr), dev(g.col_idx), seed=5).colors.cpu().numpy()
    c = pgc.pgc_color_pd2(b.n_rows, b.n_cols, dev(b.row_ptr), dev(b.col_idx), dev(b.col_ptr),
                          dev(b.row_idx), seed=5).colors.cpu().numpy()
    assert np.array_equal(a, c)


def test_host_loop_and_geometry(pgc):
    g = gen.stencil3d(9, 9, 9, points=27)
    d2_parity(pgc, g, flags=pgc.PGC_HOST_LOOP)
    for block, per_sm in ((128, 1), (512, 2), (1024, 1)):
        d2_parity(pgc, g, seed=2, block=block, grid_per_sm=per_sm)
    b = gen.bipartite(5000, 2000, seed=3)
    pd2_parity(pgc, b, flags=pgc.PGC_HOST_LOOP)


def test_host_arrays_and_edge_cases(pgc):
    g = gen.stencil3d(6, 6, 6, points=27)
    r = pgc.pgc_color_d2(g.row_ptr, g.col_idx, seed=1)
    assert np.array_equal(r.colors, oracle.color_d2(g.row_ptr, g.col_idx).colors)
    b = gen.bipartite(300, 100, seed=1)
    r = pgc.pgc_color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx)
    want = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx)
    assert np.array_equal(r.colors, want.colors)
    # edgeless, n = 0, empty rows and isolated columns
    d2_parity(pgc, gen.empty(50))
    r = pgc.pgc_color_d2(np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert r.rounds == 0 and r.num_colors == 0
    rows = [[0, 2], [], [2, 3], []]
    b = _graphs.bipartite_from_rows(rows, 6)     # columns 1, 4, 5 are in no row
    pd2_parity(pgc, b)
    # PD2 with CSR/CSC that disagree is rejected
    with pytest.raises(pgc.PgcError):
        pgc.pgc_color_pd2(2, 2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32),
                          np.array([0, 1, 1], np.int32), np.array([0], np.int32))
