"""Pins for the CPU oracle: facts fixed by the paper and by mathematics, not
by the oracle itself (published hash vectors, hand-worked examples, closed
forms, invariants, reductions between the three problems, brute force)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import setbased
from paper_2107_00075_gb300 import inputs as gen
from tests import _graphs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def h(v, seed=1):
    return oracle.splitmix64(seed ^ v)


# ----------------------------------------------------------------- hash ---
def test_splitmix64_published_vector():
    """splitmix64 from state 0 (Steele et al. 2014; Vigna's splitmix64.c)."""
    gamma = 0x9E3779B97F4A7C15
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for k, want in rows:
        state = ((int(k) - 1) * gamma) % 2**64
        assert oracle.splitmix64(state) == int(want, 16)
        assert setbased.splitmix64(state) == int(want, 16)


# --------------------------------------------------------- Alg. 4 order ---
def test_alg4_decision_order():
    R = oracle.v_is_recolored
    # lower degree is recolored, whatever the random numbers and ids
    assert R(3, 1, 0, 5, 2**63, 9) is True
    assert R(5, 2**63, 9, 3, 1, 0) is False
    # equal degree: the higher random number is recolored
    assert R(4, 100, 0, 4, 50, 9) is True
    assert R(4, 50, 9, 4, 100, 0) is False
    # random numbers compared as unsigned 64-bit
    assert R(4, 2**63 + 1, 1, 4, 5, 2) is True
    # equal degree and random number: the higher id is recolored
    assert R(4, 7, 9, 4, 7, 3) is True
    assert R(4, 7, 3, 4, 7, 9) is False
    # recolorDegrees off: degree ignored
    assert R(3, 100, 0, 5, 50, 9, recolor_degrees=False) is True
    assert R(5, 50, 9, 3, 100, 0, recolor_degrees=False) is False


def test_hash_is_injective_on_ids():
    """splitmix64 is a bijection of 64-bit words, so the id tie-break of
    Alg. 4 is never reached for distinct vertices: check on a range."""
    vals = {h(v) for v in range(20000)}
    assert len(vals) == 20000


# ------------------------------------------------------- worked examples ---
def _run_case(case, impl):
    kind = case["kind"]
    if kind == "pd2":
        rows = case["rows"]
        b = _graphs.bipartite_from_rows(rows, case["n_cols"])
        if impl == "c":
            r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                 b.row_idx, seed=case["seed"],
                                 recolor_degrees=case["recolor_degrees"])
            return list(r.colors), r.rounds, r.num_colors
        c, rounds, k, _ = setbased.color("pd2", b.row_ptr, b.col_idx, case["seed"],
                                         case["recolor_degrees"], b.col_ptr, b.row_idx)
        return c, rounds, k
    g = gen.from_edge_list(case["n"], case["edges"])
    if impl == "c":
        f = oracle.color_d1 if kind == "d1" else oracle.color_d2
        r = f(g.row_ptr, g.col_idx, seed=case["seed"], recolor_degrees=case["recolor_degrees"])
        return list(r.colors), r.rounds, r.num_colors
    c, rounds, k, _ = setbased.color(kind, g.row_ptr, g.col_idx, case["seed"],
                                     case["recolor_degrees"])
    return c, rounds, k


CASES = json.load(open(os.path.join(GOLDEN, "worked_examples.json")))["cases"]


@pytest.mark.parametrize("impl", ["c", "sets"])
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_worked_examples(case, impl):
    colors, rounds, k = _run_case(case, impl)
    assert colors == case["colors"]
    assert rounds == case["rounds"]
    assert k == case["num_colors"]


def test_worked_example_hash_order():
    """The worked examples rely on this order of rand(v) for seed 1."""
    order = sorted(range(6), key=lambda v: h(v))
    assert order == [2, 4, 5, 0, 3, 1]


# ---------------------------------------------------------- closed forms ---
@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33])
@pytest.mark.parametrize("seed", [1, 12345])
def test_complete_graph(n, seed):
    """K_n: equal degrees, so each round exactly the remaining vertex with the
    smallest rand survives: color = 1 + rank by (rand, id), rounds = n."""
    g = gen.complete(n)
    r = oracle.color_d1(g.row_ptr, g.col_idx, seed=seed)
    rank = sorted(range(n), key=lambda v: (h(v, seed), v))
    want = np.empty(n, dtype=np.int32)
    for i, v in enumerate(rank):
        want[v] = i + 1
    assert np.array_equal(r.colors, want)
    assert r.rounds == n and r.num_colors == n
    assert list(r.trace_w) == list(range(n, 0, -1))


@pytest.mark.parametrize("m,n", [(1, 2), (2, 3), (3, 7), (5, 6)])
def test_complete_bipartite_unequal(m, n):
    """K_{m,n}, m < n: the m side has the larger degree (n > m) and keeps 1."""
    g = gen.complete_bipartite(m, n)
    r = oracle.color_d1(g.row_ptr, g.col_idx, seed=7)
    assert list(r.colors[:m]) == [1] * m
    assert list(r.colors[m:]) == [2] * n
    assert r.rounds == 2 and r.num_colors == 2


@pytest.mark.parametrize("n", [1, 2, 4, 9])
def test_complete_bipartite_equal(n):
    g = gen.complete_bipartite(n, n)
    r = oracle.color_d1(g.row_ptr, g.col_idx, seed=3)
    assert r.num_colors == 2
    assert r.rounds == 2
    assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, r.colors) == 0


@pytest.mark.parametrize("leaves", [2, 3, 10, 100])
def test_star(leaves):
    g = gen.star(leaves)
    r = oracle.color_d1(g.row_ptr, g.col_idx, seed=11)
    assert r.colors[0] == 1 and set(r.colors[1:]) == {2}
    assert r.rounds == 2


@pytest.mark.parametrize("n", [1, 5, 100])
def test_edgeless(n):
    g = gen.empty(n)
    for f in (oracle.color_d1, oracle.color_d2):
        r = f(g.row_ptr, g.col_idx)
        assert set(r.colors) == {1} and r.rounds == 1 and r.num_colors == 1


def test_zero_vertices():
    g = gen.empty(0)
    for f in (oracle.color_d1, oracle.color_d2):
        r = f(g.row_ptr, g.col_idx)
        assert r.rounds == 0 and r.num_colors == 0 and len(r.colors) == 0
    r = oracle.color_pd2(0, 0, [0], [], [0], [])
    assert r.rounds == 0 and r.num_colors == 0


def test_path_and_odd_cycle_counts():
    """Paths need 2 colors and first-fit never exceeds deg + 1 = 3; odd
    cycles need exactly 3 (chi = 3, and deg + 1 = 3 bounds first-fit)."""
    for n in (2, 3, 10, 101):
        g = gen.path(n)
        r = oracle.color_d1(g.row_ptr, g.col_idx, seed=5)
        assert 2 <= r.num_colors <= 3
        assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, r.colors) == 0
    for n in (3, 5, 9, 31):
        g = gen.cycle(n)
        r = oracle.color_d1(g.row_ptr, g.col_idx, seed=2)
        assert r.num_colors == 3
        assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, r.colors) == 0


def _rank_colors(vertices, seed, first=1):
    """Colors first, first+1, ... in increasing (rand, id) order: what a
    clique of equal-degree vertices gets, one survivor per round."""
    return {v: first + i for i, v in enumerate(sorted(vertices, key=lambda v: (h(v, seed), v)))}


@pytest.mark.parametrize("leaves", [1, 2, 5, 17])
@pytest.mark.parametrize("degree_rule", [True, False])
def test_d2_star(leaves, degree_rule):
    """D2 on K_{1,n}: every pair is within two hops, a clique of n + 1.  With
    the degree rule the center (degree n) is colored 1 in round 1 and the
    leaves follow one per round in (rand, id) order; without it all n + 1
    vertices go in (rand, id) order.  Either way n + 1 rounds."""
    g = gen.star(leaves)
    seed = 3 + leaves
    r = oracle.color_d2(g.row_ptr, g.col_idx, seed=seed, recolor_degrees=degree_rule)
    if degree_rule and leaves >= 2:
        want = {0: 1, **_rank_colors(range(1, leaves + 1), seed, first=2)}
    else:     # one leaf: both vertices have degree 1, so only rand decides
        want = _rank_colors(range(leaves + 1), seed)
    assert list(r.colors) == [want[v] for v in range(leaves + 1)]
    assert r.rounds == leaves + 1 and r.num_colors == leaves + 1
    assert list(r.trace_w) == list(range(leaves + 1, 0, -1))


@pytest.mark.parametrize("m,n", [(1, 3), (2, 5), (3, 4), (4, 4)])
def test_d2_complete_bipartite(m, n):
    """D2 on K_{m,n}: a clique of m + n.  For m < n the m side has the larger
    degree, so it takes colors 1..m (by rand) before the n side takes
    m+1..m+n; for m = n all degrees tie and rand alone orders them."""
    g = gen.complete_bipartite(m, n)
    r = oracle.color_d2(g.row_ptr, g.col_idx, seed=21)
    if m < n:
        want = {**_rank_colors(range(m), 21), **_rank_colors(range(m, m + n), 21, first=m + 1)}
    else:
        want = _rank_colors(range(m + n), 21)
    assert list(r.colors) == [want[v] for v in range(m + n)]
    assert r.rounds == m + n


@pytest.mark.parametrize("sizes", [[1], [7], [3, 1, 4, 1, 5], [2, 2, 2, 9]])
def test_pd2_disjoint_rows(sizes):
    """PD2 where rows partition the columns: every column has degree 1 and
    conflicts only inside its row, so each row is an independent clique:
    its columns get 1..|row| in (rand, id) order, all rows in parallel, and
    round r's worklist holds the columns of rank >= r of every row."""
    seed = 5
    rows, c = [], 0
    for s in sizes:
        rows.append(list(range(c, c + s)))
        c += s
    # shuffle column ids across rows so a row is not a contiguous id range
    perm = np.random.default_rng(len(sizes)).permutation(c)
    rows = [sorted(int(perm[x]) for x in row) for row in rows]
    b = _graphs.bipartite_from_rows(rows, c)
    r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                         seed=seed)
    want = {}
    for row in rows:
        want.update(_rank_colors(row, seed))
    assert list(r.colors) == [want[v] for v in range(c)]
    assert r.rounds == max(sizes) and r.num_colors == max(sizes)
    assert list(r.trace_w) == [sum(max(s - k, 0) for s in sizes) for k in range(max(sizes))]


def test_pd2_hub_column_first():
    """PD2 with one column in every row and the others in one row each: the
    hub column has the largest degree, so it is colored 1 in round 1; within
    each row the remaining columns take 2, 3, ... in (rand, id) order."""
    seed = 8
    rows = [[0, 1, 2, 3], [0, 4, 5], [0, 6]]
    b = _graphs.bipartite_from_rows(rows, 7)
    r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                         seed=seed)
    want = {0: 1}
    for row in rows:
        want.update(_rank_colors(row[1:], seed, first=2))
    assert list(r.colors) == [want[v] for v in range(7)]
    assert r.rounds == 4


# ------------------------------------------------------------- invariants ---
def _random_graphs():
    out = []
    for i in range(30):
        n = 5 + (i * 7) % 60
        out.append(gen.random_small(n, 0.05 + 0.3 * ((i * 13) % 10) / 10, seed=100 + i))
    out.append(gen.stencil3d(6, 5, 4, points=7))
    out.append(gen.stencil3d(5, 4, 3, points=27))
    out.append(gen.rmat(9, 8, seed=3))
    out.append(gen.er(300, 12.0, seed=4))
    return out


def _check_trace(r, n):
    assert r.trace_w[0] == n
    assert all(a > b for a, b in zip(r.trace_w, r.trace_w[1:])), "worklist must shrink"


@pytest.mark.parametrize("idx", range(34))
def test_invariants_d1_d2(idx):
    g = _random_graphs()[idx]
    deg = np.diff(g.row_ptr)
    for kind, f in ((oracle.D1, oracle.color_d1), (oracle.D2, oracle.color_d2)):
        r = f(g.row_ptr, g.col_idx, seed=idx + 1)
        assert oracle.count_improper(kind, g.row_ptr, g.col_idx, r.colors) == 0
        assert oracle.count_non_grundy(kind, g.row_ptr, g.col_idx, r.colors) == 0
        assert r.num_colors == (r.colors.max() if g.n else 0)
        # number of distinct colors equals the maximum (Grundy)
        assert len(set(r.colors.tolist())) == r.num_colors
        _check_trace(r, g.n)
        if kind == oracle.D1:
            assert np.all(r.colors <= deg + 1)          # first-fit bound
        else:
            S = setbased.neighborhoods("d2", g.row_ptr, g.col_idx)
            assert all(r.colors[v] <= len(S[v]) + 1 for v in range(g.n))
            assert r.num_colors <= deg.max() ** 2 + 1


def test_round1_survivors_are_local_maxima():
    """Round 1 gives everyone color 1; exactly the vertices whose key beats
    all neighbors keep it (an independent set)."""
    for seed, g in enumerate(_random_graphs()[:12]):
        deg = np.diff(g.row_ptr)
        adj = _graphs.adjacency(g)
        key = lambda v: (deg[v], -h(v, seed + 1), -v)
        local_max = [v for v in range(g.n) if all(key(v) > key(u) for u in adj[v])]
        r = oracle.color_d1(g.row_ptr, g.col_idx, seed=seed + 1)
        survivors = g.n - (r.trace_w[1] if r.rounds > 1 else 0)
        assert survivors == len(local_max)
        assert all(r.colors[v] == 1 for v in local_max)


def test_stencil27_d2_lower_bound():
    """A 3x3x3 block of the 27-point stencil is a distance-2 clique."""
    g = gen.stencil3d(7, 7, 7, points=27)
    r = oracle.color_d2(g.row_ptr, g.col_idx)
    assert r.num_colors >= 27
    assert oracle.count_improper(oracle.D2, g.row_ptr, g.col_idx, r.colors) == 0


def test_stencil7_d1_bipartite_lower_bound():
    g = gen.stencil3d(8, 8, 8, points=7)
    r = oracle.color_d1(g.row_ptr, g.col_idx)
    assert 2 <= r.num_colors <= 7


# ------------------------------------------------------------ brute force ---
def test_brute_force_chromatic_lower_bound():
    for i in range(40):
        n = 4 + i % 9
        g = gen.random_small(n, 0.2 + 0.6 * ((i * 7) % 10) / 10, seed=1000 + i)
        chi = _graphs.chromatic_number(g)
        r = oracle.color_d1(g.row_ptr, g.col_idx, seed=i)
        assert r.num_colors >= chi
        assert r.num_colors <= max(np.diff(g.row_ptr).max(initial=0) + 1, 1)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_mycielski_lower_bound(k):
    """Mycielski graphs M_k have chromatic number k (textbook construction);
    the paper's single-GPU runs on the largest ones used chi or chi+1."""
    g = gen.mycielski(k)
    if g.n <= 12:
        assert _graphs.chromatic_number(g) == k
    r = oracle.color_d1(g.row_ptr, g.col_idx)
    assert r.num_colors >= k
    assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, r.colors) == 0


# ------------------------------------------------------------- reductions ---
@pytest.mark.parametrize("i", range(12))
def test_d2_equals_d1_on_square_without_degree_rule(i):
    """Distance-2 coloring of G is distance-1 coloring of G^2; with the
    degree term off the keys coincide, so the results must be identical."""
    g = gen.random_small(8 + 3 * i, 0.08 + 0.02 * i, seed=500 + i)
    g2 = _graphs.square(g)
    a = oracle.color_d2(g.row_ptr, g.col_idx, seed=i + 2, recolor_degrees=False)
    b = oracle.color_d1(g2.row_ptr, g2.col_idx, seed=i + 2, recolor_degrees=False)
    assert np.array_equal(a.colors, b.colors) and a.rounds == b.rounds


@pytest.mark.parametrize("i", range(12))
def test_d2_equals_pd2_on_closed_neighborhoods(i):
    """Rows N[u] as nets: two vertices share a net iff they are within two
    hops, and the column degree |{u : v in N[u]}| = deg(v) + 1 orders keys
    like deg(v).  So PD2 on that matrix equals D2 on G, degree rule on."""
    g = gen.random_small(8 + 3 * i, 0.08 + 0.02 * i, seed=700 + i)
    b = _graphs.closed_neighborhood_matrix(g)
    a = oracle.color_d2(g.row_ptr, g.col_idx, seed=i + 9)
    c = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                         seed=i + 9)
    assert np.array_equal(a.colors, c.colors) and a.rounds == c.rounds


@pytest.mark.parametrize("i", range(12))
def test_pd2_equals_d1_on_column_intersection_without_degree_rule(i):
    b = gen.random_bipartite_small(6 + i, 5 + 2 * i, 0.15, seed=900 + i)
    g = _graphs.column_intersection(b)
    a = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                         seed=i + 4, recolor_degrees=False)
    c = oracle.color_d1(g.row_ptr, g.col_idx, seed=i + 4, recolor_degrees=False)
    assert np.array_equal(a.colors, c.colors) and a.rounds == c.rounds
    assert oracle.count_improper(oracle.PD2, b.row_ptr, b.col_idx, a.colors,
                                 n_rows=b.n_rows, n_cols=b.n_cols, col_ptr=b.col_ptr,
                                 row_idx=b.row_idx) == 0
    assert oracle.count_non_grundy(oracle.PD2, b.row_ptr, b.col_idx, a.colors,
                                   n_rows=b.n_rows, n_cols=b.n_cols, col_ptr=b.col_ptr,
                                   row_idx=b.row_idx) == 0


def test_pd2_lower_bound_row_length():
    b = gen.bipartite(400, 150, seed=3)
    r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx)
    assert r.num_colors >= np.diff(b.row_ptr).max()
    assert oracle.count_improper(oracle.PD2, b.row_ptr, b.col_idx, r.colors,
                                 n_rows=b.n_rows, n_cols=b.n_cols, col_ptr=b.col_ptr,
                                 row_idx=b.row_idx) == 0


# --------------------------------------------- cross-check vs set version ---
def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield gen.from_edge_list(n, [p for j, p in enumerate(pairs) if mask >> j & 1])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_exhaustive_small_graphs_match_set_version(n):
    for g in _all_graphs(n):
        for kind, f in (("d1", oracle.color_d1), ("d2", oracle.color_d2)):
            for rd in (True, False):
                r = f(g.row_ptr, g.col_idx, seed=n, recolor_degrees=rd)
                c, rounds, k, sizes = setbased.color(kind, g.row_ptr, g.col_idx, n, rd)
                assert list(r.colors) == c and r.rounds == rounds and r.num_colors == k
                assert list(r.trace_w) == sizes


@pytest.mark.parametrize("n_rows,n_cols", [(1, 4), (2, 3), (2, 5), (3, 3), (3, 4), (4, 3)])
def test_exhaustive_small_patterns_match_set_version(n_rows, n_cols):
    """Every rows x columns pattern of the given shape (all 2^(rows*cols)
    of them), with and without the degree rule."""
    cells = [(r, c) for r in range(n_rows) for c in range(n_cols)]
    for mask in range(1 << len(cells)):
        rows = [[c for (r2, c) in cells if r2 == r and mask >> cells.index((r2, c)) & 1]
                for r in range(n_rows)]
        b = _graphs.bipartite_from_rows(rows, n_cols)
        for rd in (True, False):
            r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                 b.row_idx, seed=mask + 1, recolor_degrees=rd)
            c, rounds, k, sizes = setbased.color("pd2", b.row_ptr, b.col_idx, mask + 1, rd,
                                                 b.col_ptr, b.row_idx)
            assert list(r.colors) == c and r.rounds == rounds and r.num_colors == k
            assert list(r.trace_w) == sizes


def test_random_graphs_match_set_version():
    """10^4 random cases with n <= 12: 8000 graphs (D1 and D2) and 2000
    row x column patterns (PD2), seeds and the degree flag varied."""
    rng = np.random.default_rng(42)
    for i in range(8000):
        n = int(rng.integers(1, 13))
        g = gen.random_small(n, float(rng.uniform(0.05, 0.9)), seed=int(rng.integers(1 << 30)))
        seed = int(rng.integers(1 << 62))
        for kind, f in (("d1", oracle.color_d1), ("d2", oracle.color_d2)):
            rd = bool(i % 3)
            r = f(g.row_ptr, g.col_idx, seed=seed, recolor_degrees=rd)
            c, rounds, k, sizes = setbased.color(kind, g.row_ptr, g.col_idx, seed, rd)
            assert list(r.colors) == c and r.rounds == rounds and list(r.trace_w) == sizes
    for i in range(2000):
        b = gen.random_bipartite_small(int(rng.integers(1, 10)), int(rng.integers(1, 12)),
                                       float(rng.uniform(0.05, 0.6)), seed=i)
        seed = int(rng.integers(1 << 62))
        rd = bool(i % 2)
        r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                             seed=seed, recolor_degrees=rd)
        c, rounds, k, sizes = setbased.color("pd2", b.row_ptr, b.col_idx, seed, rd,
                                             b.col_ptr, b.row_idx)
        assert list(r.colors) == c and r.rounds == rounds and list(r.trace_w) == sizes


# --------------------------------------------------------- argument checks ---
def test_rejects_bad_csr():
    with pytest.raises(RuntimeError):
        oracle.color_d1([0, 2, 1], [1, 0])          # row_ptr not monotone
    with pytest.raises(RuntimeError):
        oracle.color_d1([0, 1, 2], [1, 5])          # id out of range


def test_self_loops_and_duplicates_tolerated():
    """u == v is skipped as a neighbor (it still counts in the degree)."""
    rp = np.array([0, 3, 5, 6], dtype=np.int32)
    ci = np.array([0, 1, 1, 0, 2, 1], dtype=np.int32)   # 0: {0,1,1}; 1: {0,2}; 2: {1}
    r = oracle.color_d1(rp, ci)
    assert oracle.count_improper(oracle.D1, rp, ci, r.colors) == 0
    # vertex 0 has degree 3 (self-loop and duplicate counted) > deg(1) = 2
    assert r.colors[0] == 1


# ---------------------------------------------------------------- checkers ---
def test_checkers_on_hand_colorings():
    """The properness and Grundy checkers against colorings checked by hand."""
    g = gen.path(3)                       # 0 - 1 - 2
    D1 = oracle.D1
    assert oracle.count_improper(D1, g.row_ptr, g.col_idx, [1, 2, 1]) == 0
    assert oracle.count_improper(D1, g.row_ptr, g.col_idx, [1, 1, 2]) == 2   # (0,1) and (1,0)
    assert oracle.count_improper(D1, g.row_ptr, g.col_idx, [1, 0, 1]) == 1   # uncolored vertex
    assert oracle.count_non_grundy(D1, g.row_ptr, g.col_idx, [2, 1, 2]) == 0
    assert oracle.count_non_grundy(D1, g.row_ptr, g.col_idx, [1, 2, 3]) == 1  # 2 sees only 2
    assert oracle.count_non_grundy(D1, g.row_ptr, g.col_idx, [3, 1, 2]) == 1  # 0 sees only 1
    # distance 2: on the path every pair is within two hops
    assert oracle.count_improper(oracle.D2, g.row_ptr, g.col_idx, [2, 1, 2]) == 2
    assert oracle.count_improper(oracle.D2, g.row_ptr, g.col_idx, [3, 1, 2]) == 0
    assert oracle.count_non_grundy(oracle.D2, g.row_ptr, g.col_idx, [3, 1, 2]) == 0
    # partial distance 2: rows {0,1} and {1,2}; columns 0 and 2 share no row
    b = _graphs.bipartite_from_rows([[0, 1], [1, 2]], 3)
    kw = dict(n_rows=2, n_cols=3, col_ptr=b.col_ptr, row_idx=b.row_idx)
    assert oracle.count_improper(oracle.PD2, b.row_ptr, b.col_idx, [2, 1, 2], **kw) == 0
    assert oracle.count_improper(oracle.PD2, b.row_ptr, b.col_idx, [1, 1, 2], **kw) == 2
    assert oracle.count_non_grundy(oracle.PD2, b.row_ptr, b.col_idx, [2, 1, 2], **kw) == 0
    assert oracle.count_non_grundy(oracle.PD2, b.row_ptr, b.col_idx, [3, 1, 2], **kw) == 1  # column 0


# ------------------------------------------- per-round degree sums (trace_s) ---
# trace_s[r-1] is S_r = the sum of deg(v) over the worklist W_r of round r
# (the degree of Sec. 3.3: row length for D1/D2, column length for PD2).
# These pins fix it from closed forms, independently of the oracle's loop.
@pytest.mark.parametrize("n", [1, 2, 5, 16])
def test_trace_s_complete_graph(n):
    """K_n: W_r holds n - r + 1 vertices, each of degree n - 1."""
    g = gen.complete(n)
    r = oracle.color_d1(g.row_ptr, g.col_idx, seed=4)
    assert list(r.trace_s) == [(n - 1) * (n - k) for k in range(n)]


@pytest.mark.parametrize("leaves", [2, 3, 10])
def test_trace_s_star(leaves):
    """Star K_{1,n}: round 1 holds every vertex (n + n * 1 = 2n), round 2 the
    n leaves (degree 1 each)."""
    g = gen.star(leaves)
    r = oracle.color_d1(g.row_ptr, g.col_idx, seed=11)
    assert list(r.trace_w) == [leaves + 1, leaves]
    assert list(r.trace_s) == [2 * leaves, leaves]


@pytest.mark.parametrize("m,n", [(1, 2), (3, 7), (5, 6)])
def test_trace_s_complete_bipartite(m, n):
    """K_{m,n}, m < n: round 1 all m + n vertices (2mn), round 2 the n side,
    each of degree m."""
    g = gen.complete_bipartite(m, n)
    r = oracle.color_d1(g.row_ptr, g.col_idx, seed=7)
    assert list(r.trace_s) == [2 * m * n, n * m]


@pytest.mark.parametrize("leaves", [2, 5, 17])
def test_trace_s_d2_star(leaves):
    """D2 on K_{1,n} with the degree rule: round 1 holds all n + 1 vertices
    (2n), then the leaves leave one per round; the sum is of 1-hop degrees
    (1 per leaf), not of two-hop neighborhood sizes (n per leaf)."""
    g = gen.star(leaves)
    r = oracle.color_d2(g.row_ptr, g.col_idx, seed=3 + leaves)
    assert list(r.trace_s) == [2 * leaves] + list(range(leaves, 0, -1))


@pytest.mark.parametrize("sizes", [[7], [3, 1, 4, 1, 5]])
def test_trace_s_pd2_disjoint_rows(sizes):
    """PD2 with rows partitioning the columns: every column has degree 1, so
    S_r = |W_r| = the columns of rank >= r within their row."""
    rows, c = [], 0
    for s in sizes:
        rows.append(list(range(c, c + s)))
        c += s
    b = _graphs.bipartite_from_rows(rows, c)
    r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                         seed=5)
    want = [sum(max(s - k, 0) for s in sizes) for k in range(max(sizes))]
    assert list(r.trace_s) == want


def test_trace_s_pd2_hub_column():
    """Hub column 0 in all three rows (degree 3) plus columns of degree 1: the
    hub wins round 1, so S_1 = 3 + 6 and S_r = |W_r| afterwards."""
    rows = [[0, 1, 2, 3], [0, 4, 5], [0, 6]]
    b = _graphs.bipartite_from_rows(rows, 7)
    r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                         seed=8)
    assert r.trace_s[0] == 9
    assert list(r.trace_s[1:]) == list(r.trace_w[1:])


@pytest.mark.parametrize("i", range(12))
def test_trace_s_matches_set_version_worklists(i):
    """On random graphs: the degree sum over each round's worklist, with the
    worklists taken from the set-based restatement."""
    g = gen.random_small(6 + i, 0.35, seed=300 + i)
    deg = np.diff(g.row_ptr)
    for kind, f in (("d1", oracle.color_d1), ("d2", oracle.color_d2)):
        r = f(g.row_ptr, g.col_idx, seed=i + 2)
        lists = setbased.worklists(kind, g.row_ptr, g.col_idx, i + 2, True)
        assert list(r.trace_w) == [len(w) for w in lists]
        assert list(r.trace_s) == [int(sum(deg[w])) for w in lists]
