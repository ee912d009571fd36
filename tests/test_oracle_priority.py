"""Pins for the oracle's round-varying priorities (Sec. 3.3, closing
paragraph: a "dynamic" degree based on how many neighbors have been colored,
and the "saturation degree", how many colors the colored neighbors hold), D1.
Readings: both are taken at the start of each round; dynamic = adjacency
entries whose vertex is still uncolored; saturation = distinct colors
1..deg(v)+1 among colored neighbors.  They replace deg() in Alg. 4."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import setbased
from paper_2107_00075_gb300 import inputs as gen

DYN, SAT = oracle.PRIO_DYNAMIC, oracle.PRIO_SATURATION


def h(v, seed):
    return setbased.splitmix64((seed ^ v) & setbased.MASK64)


def test_worked_example_dynamic_degree():
    """Edges 0-1 0-4 0-5 1-2 1-3 2-3 2-4, seed 1.  Degrees 3 3 3 2 2 1; rand
    order (smallest first) 2 4 5 0 3 1.
    Round 1 (all tentative 1; dynamic = static degree): 0 beats 1 (equal
    degree, smaller rand) and nothing beats 0; 2 beats 1, 3 and 4; so 0 and 2
    keep 1 and 1, 3, 4, 5 go on.
    Round 2: first fit gives 1, 3, 4, 5 color 2.  The 1-3 conflict decides it:
    static degrees 3 > 2, so 3 is recolored and ends at 3 in round 3 ->
    colors 1 2 1 3 2 2.  Dynamic degrees: 1 has one uncolored neighbor (3),
    3 has one (1); the tie goes to rand, smaller for 3, so 1 is recolored
    and takes 3 in round 3 -> colors 1 3 1 2 2 2."""
    g = gen.from_edge_list(6, [(0, 1), (0, 4), (0, 5), (1, 2), (1, 3), (2, 3), (2, 4)])
    assert sorted(range(6), key=lambda v: h(v, 1)) == [2, 4, 5, 0, 3, 1]
    s = oracle.color_d1(g.row_ptr, g.col_idx, seed=1)
    d = oracle.color_d1_priority(g.row_ptr, g.col_idx, DYN, seed=1)
    assert list(s.colors) == [1, 2, 1, 3, 2, 2] and s.rounds == 3
    assert list(d.colors) == [1, 3, 1, 2, 2, 2] and d.rounds == 3
    assert list(d.trace_w) == [6, 4, 1]


@pytest.mark.parametrize("leaves,seed", [(4, 3), (6, 2), (9, 5), (12, 8)])
def test_saturation_star(leaves, seed):
    """Star: in round 1 every saturation is 0, so rand alone decides.  If the
    center has the smallest rand it keeps 1 and the leaves take 2.  Otherwise
    the center loses, the leaves with a smaller rand than the center keep 1,
    the others lose to the center; in round 2 the center takes 2 and the rest
    of the leaves take 1 without conflict: 2 rounds either way."""
    g = gen.star(leaves)
    r = oracle.color_d1_priority(g.row_ptr, g.col_idx, SAT, seed=seed)
    hc = h(0, seed)
    if hc < min(h(v, seed) for v in range(1, leaves + 1)):
        want = [1] + [2] * leaves
    else:
        want = [2] + [1] * leaves
    assert list(r.colors) == want and r.rounds == 2
    n_first = sum(1 for v in range(1, leaves + 1) if h(v, seed) < hc)
    if want[0] == 2:
        assert list(r.trace_w) == [leaves + 1, leaves + 1 - n_first]


def test_saturation_star_cases_cover_both_outcomes():
    outcomes = set()
    for leaves, seed in [(4, 3), (6, 2), (9, 5), (12, 8)]:
        hc = h(0, seed)
        outcomes.add(hc < min(h(v, seed) for v in range(1, leaves + 1)))
    assert outcomes == {True, False}


@pytest.mark.parametrize("mode", [DYN, SAT])
@pytest.mark.parametrize("n", [2, 5, 13])
def test_complete_graph(mode, n):
    """K_n: every remaining vertex has the same dynamic degree and the same
    saturation, so rand decides: color = 1 + rank by rand, n rounds."""
    g = gen.complete(n)
    r = oracle.color_d1_priority(g.row_ptr, g.col_idx, mode, seed=6)
    rank = sorted(range(n), key=lambda v: (h(v, 6), v))
    assert [int(r.colors[v]) for v in rank] == list(range(1, n + 1))
    assert r.rounds == n


def _graphs():
    out = [gen.random_small(8 + i, 0.3, seed=500 + i) for i in range(12)]
    out += [gen.rmat(9, 8, seed=3), gen.er(400, 10.0, seed=2), gen.stencil3d(6, 5, 4, points=7)]
    return out


@pytest.mark.parametrize("idx", range(15))
def test_round_one_and_invariants(idx):
    g = _graphs()[idx]
    deg = np.diff(g.row_ptr)
    st = oracle.color_d1(g.row_ptr, g.col_idx, seed=idx)
    base = oracle.color_d1(g.row_ptr, g.col_idx, seed=idx, recolor_degrees=False)
    for mode, ref in ((DYN, st), (SAT, base)):
        r = oracle.color_d1_priority(g.row_ptr, g.col_idx, mode, seed=idx)
        # round 1: the dynamic degree is the degree; every saturation is 0
        # (the degree-blind rule)
        if len(ref.trace_w) > 1 and len(r.trace_w) > 1:
            assert r.trace_w[1] == ref.trace_w[1]
        assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, r.colors) == 0
        assert oracle.count_non_grundy(oracle.D1, g.row_ptr, g.col_idx, r.colors) == 0
        assert np.all(r.colors <= deg + 1)
        assert all(a > b for a, b in zip(r.trace_w, r.trace_w[1:]))
        assert list(r.trace_s) == [int(deg[w].sum()) for w in
                                   setbased.worklists("d1", g.row_ptr, g.col_idx, idx, True,
                                                      priority="dynamic" if mode == DYN
                                                      else "saturation")]


@pytest.mark.parametrize("n", [4, 5])
def test_exhaustive_small_graphs_match_set_version(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        g = gen.from_edge_list(n, [pairs[k] for k in range(len(pairs)) if mask >> k & 1])
        for mode, name in ((DYN, "dynamic"), (SAT, "saturation")):
            r = oracle.color_d1_priority(g.row_ptr, g.col_idx, mode, seed=mask)
            c, rounds, k, sizes = setbased.color("d1", g.row_ptr, g.col_idx, mask, True,
                                                 priority=name)
            assert list(r.colors) == c and r.rounds == rounds and list(r.trace_w) == sizes


def test_random_graphs_match_set_version():
    for i in range(400):
        g = gen.random_small(6 + i % 7, 0.2 + 0.05 * (i % 6), seed=2000 + i)
        for mode, name in ((DYN, "dynamic"), (SAT, "saturation")):
            r = oracle.color_d1_priority(g.row_ptr, g.col_idx, mode, seed=i)
            c, rounds, k, sizes = setbased.color("d1", g.row_ptr, g.col_idx, i, True,
                                                 priority=name)
            assert list(r.colors) == c and r.rounds == rounds


def test_rejects_unknown_mode():
    g = gen.path(3)
    with pytest.raises(RuntimeError):
        oracle.color_d1_priority(g.row_ptr, g.col_idx, 3)
