"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the pins catch each one: a pin set that a wrong oracle also passes
would prove nothing."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import setbased
from paper_2107_00075_gb300 import inputs as gen
from tests import _graphs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# (name, original text, replacement) -- each must occur exactly once
MUTANTS = [
    ("degree_rule_reversed",
     "if (recolor_degrees && deg_v < deg_u) return 1;\n    if (recolor_degrees && deg_u < deg_v) return 0;",
     "if (recolor_degrees && deg_v > deg_u) return 1;\n    if (recolor_degrees && deg_u > deg_v) return 0;"),
    ("rand_rule_reversed",
     "if (rand_v > rand_u) return 1;\n    if (rand_u > rand_v) return 0;",
     "if (rand_v < rand_u) return 1;\n    if (rand_u < rand_v) return 0;"),
    ("two_hop_dropped",
     "if (x != v) buf[k++] = x;             /* two hops via u */",
     "(void)x;"),
    ("first_fit_starts_at_2",
     "int32_t t = 1;\n            while (forbidden[t] == stamp) t += 1;",
     "int32_t t = 2;\n            while (forbidden[t] == stamp) t += 1;"),
    ("assign_sees_tentative",
     "int32_t c = committed[buf[j]];\n                if (c > 0 && c <= n + 1) forbidden[c] = stamp;",
     "int32_t c = committed[buf[j]] > 0 ? committed[buf[j]] : tent[buf[j]];\n"
     "                if (c > 0 && c <= n + 1) forbidden[c] = stamp;"),
    ("detect_ignores_tentative",
     "int32_t cu = committed[u] > 0 ? committed[u] : tent[u];",
     "int32_t cu = committed[u];"),
    ("hash_constant_typo",
     "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;",
     "z = (z ^ (z >> 27)) * 0x94D049BB133111EDULL;"),
    ("pd2_first_row_only",
     "for (int32_t e = g->col_ptr[v]; e < g->col_ptr[v + 1]; ++e) {\n            int32_t row = g->row_idx[e];\n            for (int32_t f",
     "for (int32_t e = g->col_ptr[v]; e < g->col_ptr[v + 1] && e == g->col_ptr[v]; ++e) {\n            int32_t row = g->row_idx[e];\n            for (int32_t f"),
    ("pd2_degree_from_rows",
     "if (g->kind == KIND_PD2 || (g->kind == KIND_PD2B && v < g->n_cols))\n        return g->col_ptr[v + 1] - g->col_ptr[v];",
     "if (g->kind == KIND_PD2 || (g->kind == KIND_PD2B && v < g->n_cols))\n        return 1;"),
    ("d2_one_hop_dropped",
     "if (u != v) buf[k++] = u;                 /* one hop */",
     "(void)u;"),
    ("seed_added_not_xored",
     "return oracle_splitmix64(seed ^ (uint64_t)(uint32_t)v);",
     "return oracle_splitmix64(seed + (uint64_t)(uint32_t)v);"),
    ("winner_color_off_by_one",
     "committed[v] = tent[v];\n            }",
     "committed[v] = tent[v] + (tent[v] > 1);\n            }"),
    # the per-round degree sums (trace_s)
    ("trace_s_over_next_worklist",
     "int32_t *tmp = work; work = next; next = tmp;\n        wn = nn;",
     "int32_t *tmp = work; work = next; next = tmp;\n        wn = nn;\n"
     "        if (trace_w && r <= trace_cap) {\n"
     "            int64_t s2 = 0;\n"
     "            for (int32_t i = 0; i < wn; ++i) s2 += deg[work[i]];\n"
     "            trace_s[r - 1] = s2;\n"
     "        }"),
    ("trace_s_neighborhood_size",
     "for (int32_t i = 0; i < wn; ++i) s += deg[work[i]];",
     "for (int32_t i = 0; i < wn; ++i) s += neighborhood(g, work[i], buf);"),
    # PD2 over every vertex of the bipartite graph
    ("pd2b_rows_side_local_ids",
     "rnd[v] = rand_of(seed, v);",
     "rnd[v] = rand_of(seed, (g->kind == KIND_PD2B && v >= g->n_cols) ? v - g->n_cols : v);"),
    ("pd2b_row_degree_wrong",
     "return g->row_ptr[v - g->n_cols + 1] - g->row_ptr[v - g->n_cols];",
     "return 1;"),
    ("pd2b_row_neighbors_as_column_ids",
     "if (r != i) buf[k++] = g->n_cols + r;",
     "if (r != i) buf[k++] = r;"),
    # round-varying priorities (Sec. 3.3, closing paragraph)
    ("dynamic_counts_colored_neighbors",
     "if (committed[g->col_idx[e]] == 0) p += 1;",
     "if (committed[g->col_idx[e]] != 0) p += 1;"),
    ("saturation_not_distinct",
     "if (u != v && c > 0 && c <= deg[v] + 1 && mark[c] != *stamp) {",
     "if (u != v && c > 0 && c <= deg[v] + 1) {"),
    ("trace_s_skips_first_entry",
     "for (int32_t i = 0; i < wn; ++i) s += deg[work[i]];",
     "for (int32_t i = 1; i < wn; ++i) s += deg[work[i]];"),
]


def h(v, seed):
    return setbased.splitmix64((seed ^ v) & setbased.MASK64)


def _pins_pass(lib) -> bool:
    """A compact run of the pins in test_oracle_pins.py against lib."""
    try:
        gamma = 0x9E3779B97F4A7C15
        for k, want in ((1, 0xE220A8397B1DCDAF), (2, 0x6E789E6AA1B965F4)):
            if oracle.splitmix64((k - 1) * gamma % 2**64, lib=lib) != want:
                return False
        cases = json.load(open(os.path.join(GOLDEN, "worked_examples.json")))["cases"]
        for c in cases:
            if c["kind"] == "pd2":
                b = _graphs.bipartite_from_rows(c["rows"], c["n_cols"])
                r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                     b.row_idx, seed=c["seed"],
                                     recolor_degrees=c["recolor_degrees"], lib=lib)
            else:
                g = gen.from_edge_list(c["n"], c["edges"])
                f = oracle.color_d1 if c["kind"] == "d1" else oracle.color_d2
                r = f(g.row_ptr, g.col_idx, seed=c["seed"],
                      recolor_degrees=c["recolor_degrees"], lib=lib)
            if list(r.colors) != c["colors"] or r.rounds != c["rounds"]:
                return False
        # per-round degree sums: K_n, D2 on a star, PD2 with disjoint rows
        for n in (2, 5, 9):
            g = gen.complete(n)
            r = oracle.color_d1(g.row_ptr, g.col_idx, seed=4, lib=lib)
            if list(r.trace_s) != [(n - 1) * (n - k) for k in range(n)]:
                return False
        g = gen.star(6)
        r = oracle.color_d2(g.row_ptr, g.col_idx, seed=9, lib=lib)
        if list(r.trace_s) != [12, 6, 5, 4, 3, 2, 1]:
            return False
        b = _graphs.bipartite_from_rows([[0, 1, 2], [3, 4], [5]], 6)
        r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                             seed=5, lib=lib)
        if list(r.trace_s) != [6, 3, 1]:
            return False
        # round-varying priorities: the worked example (dynamic), a star
        # (saturation), and the set-based restatement on random graphs
        g = gen.from_edge_list(6, [(0, 1), (0, 4), (0, 5), (1, 2), (1, 3), (2, 3), (2, 4)])
        r = oracle.color_d1_priority(g.row_ptr, g.col_idx, 1, seed=1, lib=lib)
        if list(r.colors) != [1, 3, 1, 2, 2, 2]:
            return False
        g = gen.star(6)
        r = oracle.color_d1_priority(g.row_ptr, g.col_idx, 2, seed=2, lib=lib)
        if list(r.colors) != [2] + [1] * 6:
            return False
        for i in range(150):
            g = gen.random_small(6 + i % 7, 0.25 + 0.05 * (i % 5), seed=7000 + i)
            for mode, name in ((1, "dynamic"), (2, "saturation")):
                r = oracle.color_d1_priority(g.row_ptr, g.col_idx, mode, seed=i, lib=lib)
                c, rounds, k, _ = setbased.color("d1", g.row_ptr, g.col_idx, i, True,
                                                 priority=name)
                if list(r.colors) != c or r.rounds != rounds:
                    return False
        # PD2 over all of B: the complete 3 x 4 pattern (both sides cliques,
        # ranked by rand of their GIDs) and a hub row
        # (with seed 1 the rows' ranks by GID 4..8 differ from those by 0..4)
        b = _graphs.bipartite_from_rows([[0, 1, 2, 3]] * 5, 4)
        r = oracle.color_pd2_bipartite(5, 4, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                                       seed=1, lib=lib)
        rank = lambda ids: {v: 1 + i for i, v in enumerate(sorted(ids, key=lambda v: (h(v, 1), v)))}
        cols, rows = rank(range(4)), rank(range(4, 9))
        if list(r.colors) != [cols[v] for v in range(4)] + [rows[v] for v in range(4, 9)]:
            return False
        b = _graphs.bipartite_from_rows([[0, 1, 2, 3], [0], [1], [2], [3]], 4)
        r = oracle.color_pd2_bipartite(5, 4, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                                       seed=2, lib=lib)   # rand ranks the hub row last
        if r.colors[4] != 1 or set(r.colors[5:]) != {2}:
            return False
        # K_{m,n} closed form and the D2 = D1(G^2) reduction
        g = gen.complete_bipartite(3, 7)
        r = oracle.color_d1(g.row_ptr, g.col_idx, seed=7, lib=lib)
        if list(r.colors) != [1] * 3 + [2] * 7:
            return False
        rng = np.random.default_rng(5)
        for i in range(40):
            g = gen.random_small(int(rng.integers(3, 12)), 0.3, seed=i)
            g2 = _graphs.square(g)
            a = oracle.color_d2(g.row_ptr, g.col_idx, seed=i, recolor_degrees=False, lib=lib)
            b = oracle.color_d1(g2.row_ptr, g2.col_idx, seed=i, recolor_degrees=False,
                                lib=lib)
            if not np.array_equal(a.colors, b.colors):
                return False
            for kind, f in (("d1", oracle.color_d1), ("d2", oracle.color_d2)):
                r = f(g.row_ptr, g.col_idx, seed=i, lib=lib)
                c, rounds, k, _ = setbased.color(kind, g.row_ptr, g.col_idx, i, True)
                if list(r.colors) != c or r.rounds != rounds:
                    return False
        for i in range(30):
            b = gen.random_bipartite_small(6, 8, 0.3, seed=i)
            r = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr,
                                 b.row_idx, seed=i, lib=lib)
            c, rounds, k, _ = setbased.color("pd2", b.row_ptr, b.col_idx, i, True,
                                             b.col_ptr, b.row_idx)
            if list(r.colors) != c:
                return False
        return True
    except RuntimeError:
        return False


def test_unmutated_oracle_passes():
    assert _pins_pass(oracle._load())


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    lib = oracle.load_library(oracle.compile_source(src.replace(old, new),
                                                    str(tmp_path / f"{name}.so")))
    assert not _pins_pass(lib), f"pins did not catch mutant {name}"
