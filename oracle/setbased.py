"""Second, independent restatement of the round-synchronous coloring, in sets.

TEST INFRASTRUCTURE.  Written separately from ``pgc_oracle.c`` (no shared
code) so that the two can be cross-checked on many tiny graphs.  Pure Python,
for graphs of a few dozen vertices.

The neighborhood S(v) is materialised as a Python set, priorities as tuples
compared lexicographically: key(v) = (deg(v), -rand(v), -v), with the
degree term dropped when the recolorDegrees rule is off.  "u beats v" means
key(u) > key(v); that is Alg. 4 (Sec. 3.3) written as one comparison.
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """splitmix64 output for state x (Steele, Lea, Flood 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def adjacency_sets(row_ptr, col_idx):
    n = len(row_ptr) - 1
    return [set(int(u) for u in col_idx[row_ptr[v]:row_ptr[v + 1]]) - {v} for v in range(n)]


def neighborhoods(kind, row_ptr, col_idx, col_ptr=None, row_idx=None):
    """S(v) for D1 ('d1'), D2 ('d2'), PD2 ('pd2', columns) or PD2 over every
    vertex of the bipartite graph ('pd2b': the columns, then the rows as
    vertices n_cols + i)."""
    if kind == "pd2b":
        n_cols = len(col_ptr) - 1
        n_rows = len(row_ptr) - 1
        cols_of = [set(int(c) for c in col_idx[row_ptr[r]:row_ptr[r + 1]]) for r in range(n_rows)]
        rows_of = [set(col_idx_rows(col_ptr, row_idx, c)) for c in range(n_cols)]
        out = []
        for v in range(n_cols):
            s = set()
            for r in rows_of[v]:
                s |= cols_of[r]
            s.discard(v)
            out.append(s)
        for i in range(n_rows):
            s = set()
            for c in cols_of[i]:
                s |= {n_cols + r for r in rows_of[c]}
            s.discard(n_cols + i)
            out.append(s)
        return out
    if kind == "pd2":
        n_cols = len(col_ptr) - 1
        rows = [set(int(c) for c in col_idx[row_ptr[r]:row_ptr[r + 1]])
                for r in range(len(row_ptr) - 1)]
        out = []
        for v in range(n_cols):
            s = set()
            for r in col_idx_rows(col_ptr, row_idx, v):
                s |= rows[r]
            s.discard(v)
            out.append(s)
        return out
    adj = adjacency_sets(row_ptr, col_idx)
    if kind == "d1":
        return adj
    out = []
    for v, nb in enumerate(adj):
        s = set(nb)
        for u in nb:
            s |= adj[u]
        s.discard(v)
        out.append(s)
    return out


def col_idx_rows(col_ptr, row_idx, v):
    return [int(r) for r in row_idx[col_ptr[v]:col_ptr[v + 1]]]


def color(kind, row_ptr, col_idx, seed=1, recolor_degrees=True, col_ptr=None, row_idx=None,
          priority="static"):
    """Returns (colors, rounds, num_colors, worklist sizes per round).
    priority (D1): "static" (the degree, computed once), "dynamic" (adjacency
    entries whose vertex is uncolored at the start of the round) or
    "saturation" (distinct colors 1..deg+1 held by colored neighbors at the
    start of the round) -- Sec. 3.3's closing paragraph."""
    colors, lists = _rounds(kind, row_ptr, col_idx, seed, recolor_degrees, col_ptr, row_idx,
                            priority)
    return colors, len(lists), max(colors, default=0), [len(w) for w in lists]


def worklists(kind, row_ptr, col_idx, seed=1, recolor_degrees=True, col_ptr=None,
              row_idx=None, priority="static"):
    """The worklist W_r of every round r = 1, 2, ... as sorted vertex lists."""
    return _rounds(kind, row_ptr, col_idx, seed, recolor_degrees, col_ptr, row_idx,
                   priority)[1]


def _rounds(kind, row_ptr, col_idx, seed, recolor_degrees, col_ptr, row_idx,
            priority="static"):
    S = neighborhoods(kind, row_ptr, col_idx, col_ptr, row_idx)
    n = len(S)
    if kind == "pd2":
        deg = [col_ptr[v + 1] - col_ptr[v] for v in range(n)]
    elif kind == "pd2b":   # degree in the bipartite graph
        n_cols = len(col_ptr) - 1
        deg = ([col_ptr[v + 1] - col_ptr[v] for v in range(n_cols)] +
               [row_ptr[i + 1] - row_ptr[i] for i in range(n - n_cols)])
    else:
        deg = [row_ptr[v + 1] - row_ptr[v] for v in range(n)]

    final = {}
    prio = list(deg)

    def key(v):
        h = splitmix64((seed ^ v) & MASK64)
        return (prio[v], -h, -v) if recolor_degrees or priority != "static" else (-h, -v)

    def round_priority(v):
        row = [int(u) for u in col_idx[row_ptr[v]:row_ptr[v + 1]]]
        if priority == "dynamic":
            return sum(1 for u in row if u not in final)
        return len({final[u] for u in row if u != v and u in final and final[u] <= deg[v] + 1})

    todo = set(range(n))
    lists = []
    while todo:
        lists.append(sorted(todo))
        if priority != "static":
            for v in todo:
                prio[v] = round_priority(v)
        tentative = {}
        for v in todo:
            used = {final[u] for u in S[v] if u in final}
            c = 1
            while c in used:
                c += 1
            tentative[v] = c
        current = dict(final)
        current.update(tentative)
        losers = {v for v in todo
                  if any(current[u] == tentative[v] and key(u) > key(v) for u in S[v])}
        for v in todo - losers:
            final[v] = tentative[v]
        todo = losers
    colors = [final[v] for v in range(n)]
    return colors, lists
