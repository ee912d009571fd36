"""Graph transformations used by the reduction pins (pure combinatorics)."""
import numpy as np

from paper_2107_00075_gb300.inputs import CSR, Bipartite


def adjacency(g: CSR):
    return [set(int(u) for u in g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]) - {v}
            for v in range(g.n)]


def csr_from_sets(sets) -> CSR:
    rp = np.zeros(len(sets) + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(s) for s in sets])
    ci = np.array([u for s in sets for u in sorted(s)], dtype=np.int32)
    return CSR(rp, ci)


def square(g: CSR) -> CSR:
    """G^2: u ~ v iff 1 <= dist(u, v) <= 2."""
    adj = adjacency(g)
    out = []
    for v, nb in enumerate(adj):
        s = set(nb)
        for u in nb:
            s |= adj[u]
        s.discard(v)
        out.append(s)
    return csr_from_sets(out)


def closed_neighborhood_matrix(g: CSR) -> Bipartite:
    """Rows = closed neighborhoods N[u], columns = vertices of g."""
    adj = adjacency(g)
    rows = [sorted(adj[u] | {u}) for u in range(g.n)]
    return bipartite_from_rows(rows, g.n)


def bipartite_from_rows(rows, n_cols) -> Bipartite:
    n_rows = len(rows)
    rp = np.zeros(n_rows + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([c for r in rows for c in r], dtype=np.int32)
    cols = [[] for _ in range(n_cols)]
    for r, row in enumerate(rows):
        for c in row:
            cols[c].append(r)
    cp = np.zeros(n_cols + 1, dtype=np.int32)
    cp[1:] = np.cumsum([len(c) for c in cols])
    ri = np.array([r for c in cols for r in c], dtype=np.int32)
    return Bipartite(n_rows, n_cols, rp, ci, cp, ri)


def column_intersection(b: Bipartite) -> CSR:
    """Columns adjacent iff they share a row."""
    out = [set() for _ in range(b.n_cols)]
    for r in range(b.n_rows):
        row = [int(c) for c in b.col_idx[b.row_ptr[r]:b.row_ptr[r + 1]]]
        for c in row:
            out[c] |= set(row)
    for c in range(b.n_cols):
        out[c].discard(c)
    return csr_from_sets(out)


def chromatic_number(g: CSR) -> int:
    """Exact chi by backtracking (n <= 12)."""
    adj = adjacency(g)
    n = g.n
    if n == 0:
        return 0
    order = sorted(range(n), key=lambda v: -len(adj[v]))
    for k in range(1, n + 1):
        col = [0] * n

        def bt(i):
            if i == n:
                return True
            v = order[i]
            for c in range(1, k + 1):
                if all(col[u] != c for u in adj[v]):
                    col[v] = c
                    if bt(i + 1):
                        return True
                    col[v] = 0
            return False

        if bt(0):
            return k
    return n
