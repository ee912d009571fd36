"""GPU parity for partial distance-2 coloring of every vertex of the
bipartite graph (pgc_color_pd2_bipartite, Sec. 3.6): colors, rounds and color
count equal the oracle's, on hand patterns, random patterns of ragged sizes
and a pattern of the 4M x 1M recipe at 1/8 scale; at the full 4M x 1M size
the columns must equal pgc_color_pd2's (bit-exact against the oracle in the
full-size test) and the rows must be a proper Grundy coloring."""
import numpy as np
import pytest

import oracle
from paper_2107_00075_gb300 import inputs as gen
from tests import _graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pgc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2107_00075_gb300 as p
    return p


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check(pgc, b, seed=1, recolor_degrees=True, **kw):
    flags = kw.pop("flags", 0) | (0 if recolor_degrees else pgc.PGC_NO_DEGREE_RULE)
    prof = pgc.Profile(trace_cap=100000)
    r = pgc.pgc_color_pd2_bipartite(b.n_rows, b.n_cols, dev(b.row_ptr), dev(b.col_idx),
                                    dev(b.col_ptr), dev(b.row_idx), seed=seed, flags=flags,
                                    profile=prof, **kw)
    want = oracle.color_pd2_bipartite(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                      b.row_idx, seed=seed, recolor_degrees=recolor_degrees)
    got = r.colors.cpu().numpy()
    assert r.rounds == want.rounds and r.num_colors == want.num_colors
    diff = np.nonzero(got != want.colors)[0]
    assert len(diff) == 0, f"{len(diff)} colors differ, first at {diff[:5]}"
    assert np.array_equal(prof.trace_w, want.trace_w)
    assert np.array_equal(prof.trace_s, want.trace_s)


def test_hand_patterns(pgc):
    for rows, n_cols in (([[0, 2], [1, 2], [0, 1, 3]], 4), ([[0, 1, 2, 3]] * 5, 4),
                         ([[0]] * 6, 1), ([[0, 1, 2, 3], [0], [1], [2], [3]], 4),
                         ([[], [0], []], 2)):
        b = _graphs.bipartite_from_rows(rows, n_cols)
        for seed in (1, 2, 7):
            check(pgc, b, seed=seed)
            check(pgc, b, seed=seed, recolor_degrees=False)


@pytest.mark.parametrize("shape", [(31, 33), (257, 100), (1000, 3000), (5000, 700)])
def test_random_patterns(pgc, shape):
    n_rows, n_cols = shape
    b = gen.bipartite(n_rows, n_cols, lam=7.0, seed=n_rows)
    check(pgc, b, seed=3)
    check(pgc, b, seed=3, recolor_degrees=False)
    check(pgc, b, seed=5, flags=pgc.PGC_HOST_LOOP)


def test_one_eighth_of_the_bench_pattern(pgc):
    b = gen.bipartite(1 << 19, 1 << 17, lam=7.0, seed=1)
    check(pgc, b, seed=1)


def test_full_size_columns_and_rows(pgc):
    b = gen.bipartite(1 << 22, 1 << 20, lam=7.0, seed=1)
    a = [dev(x) for x in (b.row_ptr, b.col_idx, b.col_ptr, b.row_idx)]
    r = pgc.pgc_color_pd2_bipartite(b.n_rows, b.n_cols, *a, seed=1)
    p = pgc.pgc_color_pd2(b.n_rows, b.n_cols, *a, seed=1)
    got = r.colors.cpu().numpy()
    assert np.array_equal(got[:b.n_cols], p.colors.cpu().numpy())
    assert r.num_colors >= p.num_colors and r.rounds >= p.rounds
    kw = dict(n_rows=b.n_rows, n_cols=b.n_cols, col_ptr=b.col_ptr, row_idx=b.row_idx)
    assert oracle.count_improper(oracle.PD2B, b.row_ptr, b.col_idx, got, **kw) == 0
    assert oracle.count_non_grundy(oracle.PD2B, b.row_ptr, b.col_idx, got, **kw) == 0
    # the rows' largest color is at least the largest column degree (a
    # column's rows form a clique)
    assert got[b.n_cols:].max() >= np.diff(b.col_ptr).max()


def test_validate_and_empty(pgc):
    b = gen.bipartite(200, 50, seed=9)
    check(pgc, b, seed=2, flags=pgc.PGC_VALIDATE)
    ri = b.row_idx.copy()
    ri[0] = (ri[0] + 1) % b.n_rows
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_pd2_bipartite(b.n_rows, b.n_cols, dev(b.row_ptr), dev(b.col_idx),
                                    dev(b.col_ptr), dev(ri), flags=pgc.PGC_VALIDATE)
    assert e.value.status == 1
    r = pgc.pgc_color_pd2_bipartite(0, 0, dev(np.zeros(1, np.int32)), dev(np.zeros(0, np.int32)),
                                    dev(np.zeros(1, np.int32)), dev(np.zeros(0, np.int32)))
    assert r.rounds == 0 and r.num_colors == 0
