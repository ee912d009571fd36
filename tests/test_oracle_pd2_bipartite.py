"""Pins for the oracle's partial distance-2 coloring of every vertex of the
bipartite graph (Sec. 3.6: the method colors all of B(V_s, V_t, E_B), two-hop
conflicts only).  Vertices 0..n_cols-1 are the columns, n_cols + i is row i;
that index is the GID whose rand() breaks degree ties (Alg. 4)."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import setbased
from paper_2107_00075_gb300 import inputs as gen
from tests import _graphs


def h(v, seed):
    return setbased.splitmix64((seed ^ v) & setbased.MASK64)


def rank_colors(ids, seed, first=1):
    return {v: first + i for i, v in enumerate(sorted(ids, key=lambda v: (h(v, seed), v)))}


def run(rows, n_cols, seed, recolor_degrees=True):
    b = _graphs.bipartite_from_rows(rows, n_cols)
    return b, oracle.color_pd2_bipartite(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                         b.row_idx, seed=seed, recolor_degrees=recolor_degrees)


@pytest.mark.parametrize("m", [1, 2, 5, 9])
def test_one_full_row(m):
    """A single row holding all m columns: the columns form a clique of equal
    degree (colors 1..m by rand of their GIDs), the row shares no column with
    another row (color 1); m rounds."""
    seed = 3
    b, r = run([list(range(m))], m, seed)
    want = rank_colors(range(m), seed)
    assert list(r.colors[:m]) == [want[v] for v in range(m)]
    assert r.colors[m] == 1
    assert r.rounds == m and r.num_colors == m


@pytest.mark.parametrize("n_rows", [2, 3, 7])
def test_one_column_in_every_row(n_rows):
    """Every row holds only column 0: the column gets 1; the rows form a clique
    of equal degree 1, ranked by rand of their GIDs n_cols + i."""
    seed = 5
    b, r = run([[0]] * n_rows, 1, seed)
    assert r.colors[0] == 1
    want = rank_colors([1 + i for i in range(n_rows)], seed)
    assert list(r.colors[1:]) == [want[1 + i] for i in range(n_rows)]
    assert r.rounds == n_rows and r.num_colors == n_rows


@pytest.mark.parametrize("m,n", [(2, 3), (4, 4), (5, 2)])
def test_complete_pattern(m, n):
    """All m x n entries: both sides are cliques (columns of degree m, rows of
    degree n); each ranks by rand of its GIDs; rounds = the larger side."""
    seed = 11
    b, r = run([list(range(n))] * m, n, seed)
    cols = rank_colors(range(n), seed)
    rows = rank_colors([n + i for i in range(m)], seed)
    assert list(r.colors) == [cols[v] for v in range(n)] + [rows[n + i] for i in range(m)]
    assert r.rounds == max(m, n)


@pytest.mark.parametrize("k", [2, 4, 8])
def test_hub_row_keeps_color_one(k):
    """Row 0 holds every column, rows 1..k one column each: on the row side a
    star whose center (degree k) beats its leaves (degree 1) in round 1."""
    rows = [list(range(k))] + [[j] for j in range(k)]
    b, r = run(rows, k, seed=7)
    assert r.colors[k] == 1 and set(r.colors[k + 1:]) == {2}


def test_columns_equal_plain_pd2():
    """The sides never conflict (two-hop paths stay on one side), and column
    ids are the same, so the columns get exactly pgc's column-only PD2 colors."""
    for i in range(25):
        b = gen.random_bipartite_small(7, 9, 0.3, seed=40 + i)
        r = oracle.color_pd2_bipartite(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                       b.row_idx, seed=i)
        p = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                             seed=i)
        assert np.array_equal(r.colors[:b.n_cols], p.colors)
        assert r.rounds >= p.rounds


@pytest.mark.parametrize("n_rows,n_cols", [(2, 3), (3, 3), (2, 4), (3, 4)])
def test_exhaustive_small_patterns_match_set_version(n_rows, n_cols):
    cells = [(r, c) for r in range(n_rows) for c in range(n_cols)]
    for mask in range(1 << len(cells)):
        rows = [[] for _ in range(n_rows)]
        for k, (r, c) in enumerate(cells):
            if mask >> k & 1:
                rows[r].append(c)
        b = _graphs.bipartite_from_rows(rows, n_cols)
        for rd in (True, False):
            r = oracle.color_pd2_bipartite(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                           b.row_idx, seed=mask, recolor_degrees=rd)
            c, rounds, k, sizes = setbased.color("pd2b", b.row_ptr, b.col_idx, mask, rd,
                                                 b.col_ptr, b.row_idx)
            assert list(r.colors) == c and r.rounds == rounds
            assert list(r.trace_w) == sizes


def test_random_patterns_proper_and_grundy():
    for i in range(20):
        b = gen.random_bipartite_small(20, 15, 0.2, seed=300 + i)
        r = oracle.color_pd2_bipartite(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                       b.row_idx, seed=i + 1)
        kw = dict(n_rows=b.n_rows, n_cols=b.n_cols, col_ptr=b.col_ptr, row_idx=b.row_idx)
        assert oracle.count_improper(oracle.PD2B, b.row_ptr, b.col_idx, r.colors, **kw) == 0
        assert oracle.count_non_grundy(oracle.PD2B, b.row_ptr, b.col_idx, r.colors, **kw) == 0
        # a row's color is at most its two-hop neighborhood + 1
        S = setbased.neighborhoods("pd2b", b.row_ptr, b.col_idx, b.col_ptr, b.row_idx)
        assert all(r.colors[v] <= len(S[v]) + 1 for v in range(len(S)))


def test_checker_rejects_a_row_conflict():
    b = _graphs.bipartite_from_rows([[0, 1], [1, 2]], 3)
    good = [1, 2, 1, 1, 2]
    kw = dict(n_rows=2, n_cols=3, col_ptr=b.col_ptr, row_idx=b.row_idx)
    assert oracle.count_improper(oracle.PD2B, b.row_ptr, b.col_idx, good, **kw) == 0
    bad = [1, 2, 1, 1, 1]   # rows 0 and 1 share column 1
    assert oracle.count_improper(oracle.PD2B, b.row_ptr, b.col_idx, bad, **kw) == 2
