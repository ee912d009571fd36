"""The seeded input generators against their recipes: closed-form sizes of
the stencils and grids, structure (symmetric, no loops, no repeats, ids in
range, CSR and CSC of one pattern), R-MAT's id scrambling, the Poisson row
lengths of the Jacobian patterns, the batch layout, and determinism.  These
generators feed both the oracle and the CUDA path, so a wrong recipe would
go unnoticed by parity alone."""
import math

import numpy as np
import pytest

from paper_2107_00075_gb300 import inputs as gen


def _structure(g, sorted_rows=True):
    n = g.n
    rp, ci = g.row_ptr, g.col_idx
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(ci)
    assert ci.size == 0 or (ci.min() >= 0 and ci.max() < n)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    assert not np.any(src == ci), "self-loop"
    key = src * n + ci
    assert len(np.unique(key)) == len(key), "repeated entry"
    rev = np.sort(ci.astype(np.int64) * n + src)
    assert np.array_equal(np.sort(key), rev), "not symmetric"
    if sorted_rows:
        for v in range(0, n, max(1, n // 200)):
            row = ci[rp[v]:rp[v + 1]]
            assert np.all(np.diff(row) > 0)


@pytest.mark.parametrize("dims", [(32, 32, 32), (5, 4, 3), (1, 1, 7), (9, 1, 1)])
def test_stencil7_closed_form(dims):
    nx, ny, nz = dims
    g = gen.stencil3d(nx, ny, nz, points=7)
    assert g.n == nx * ny * nz
    assert g.nnz == 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1))
    _structure(g)
    # id = x + nx*(y + ny*z): the neighbors of the origin are +x, +y, +z
    want0 = sorted(v for v, ok in ((1, nx > 1), (nx, ny > 1), (nx * ny, nz > 1)) if ok)
    assert list(g.col_idx[g.row_ptr[0]:g.row_ptr[1]]) == want0


def test_stencil7_32_cubed_is_the_small_workload():
    g = gen.stencil3d(32, 32, 32, points=7)
    assert g.n == 32768 and g.nnz == 190464
    deg = np.diff(g.row_ptr)
    assert deg.min() == 3 and deg.max() == 6


@pytest.mark.parametrize("dims", [(12, 11, 10), (3, 3, 3), (2, 5, 1)])
def test_stencil27_closed_form(dims):
    nx, ny, nz = dims
    g = gen.stencil3d(nx, ny, nz, points=27)
    # ordered pairs with |dx|, |dy|, |dz| <= 1, minus the n self pairs
    assert g.nnz == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2) - nx * ny * nz
    _structure(g)
    # the D2 workload's size follows from the same count
    assert (3 * 128 - 2) ** 3 - 128 ** 3 == 53_645_816


@pytest.mark.parametrize("n", [1, 2, 100, 1000, 12345])
def test_grid2d_recipe(n):
    g = gen.grid2d(n)
    w = math.isqrt(n - 1) + 1 if n > 1 else 1     # ceil(sqrt(n))
    assert w * w >= n and (w - 1) ** 2 < n
    want = [set() for _ in range(n)]
    for v in range(n):
        if (v % w) + 1 < w and v + 1 < n:
            want[v].add(v + 1)
            want[v + 1].add(v)
        if v + w < n:
            want[v].add(v + w)
            want[v + w].add(v)
    assert g.n == n
    for v in range(n):
        assert set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) == want[v]


def test_rmat_structure_and_skew():
    g = gen.rmat(14, 16, seed=1)
    assert g.n == 1 << 14
    assert g.nnz <= 2 * 16 * (1 << 14)
    _structure(g)
    deg = np.diff(g.row_ptr)
    assert deg.max() > 20 * deg.mean()        # skewed: a few hubs
    assert np.count_nonzero(deg == 0) > 0     # isolated vertices are kept


def test_rmat_id_scrambling():
    """With every sample in quadrant b (source bit 0, destination bit 1 at
    every level) the raw edge is (0, 2^s - 1); the ids must come out as
    v' = (v * 0x9E3779B1 + 12345) mod 2^s."""
    s = 10
    g = gen.rmat(s, 4, seed=3, a=0.0, b=1.0, c=0.0)
    f = lambda v: (v * 0x9E3779B1 + 12345) % (1 << s)
    u, v = f(0), f((1 << s) - 1)
    assert g.nnz == 2
    assert list(g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]) == [v]
    assert list(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]) == [u]
    raw = gen.rmat(s, 4, seed=3, a=0.0, b=1.0, c=0.0, scramble=False)
    assert raw.nnz == 2 and list(raw.col_idx[raw.row_ptr[0]:raw.row_ptr[1]]) == [(1 << s) - 1]


def test_rmat_subrange_redraws_out_of_range_ids():
    g = gen.rmat(12, 8, seed=5, n_vertices=3000)
    assert g.n == 3000
    _structure(g)


def test_er_recipe():
    n, d = 20000, 16.0
    g = gen.er(n, d, seed=4)
    _structure(g)
    m = round(n * d / 2)
    assert 0.99 * 2 * m <= g.nnz <= 2 * m     # repeats and loops removed


def test_bipartite_recipe():
    n_rows, n_cols, lam = 200_000, 1 << 20, 7.0
    b = gen.bipartite(n_rows, n_cols, lam=lam, seed=2)
    rp, ci, cp, ri = b.row_ptr, b.col_idx, b.col_ptr, b.row_idx
    assert rp[-1] == cp[-1] == b.nnz
    length = np.diff(rp)
    assert length.min() >= 1
    # 1 + Poisson(lam): mean 1 + lam, variance lam (repeats are negligible here)
    assert abs(length.mean() - (1 + lam)) < 0.03
    assert abs(length.var() - lam) < 0.15
    # no repeated column in a row, ids in range
    r = np.repeat(np.arange(n_rows, dtype=np.int64), length)
    key = r * n_cols + ci
    assert len(np.unique(key)) == len(key)
    assert ci.min() >= 0 and ci.max() < n_cols
    # CSC is the transpose of CSR
    c = np.repeat(np.arange(n_cols, dtype=np.int64), np.diff(cp))
    assert np.array_equal(np.sort(key), np.sort(ri.astype(np.int64) * n_cols + c))
    # uniform columns: column degree ~ Poisson(nnz / n_cols)
    cdeg = np.diff(cp)
    assert abs(cdeg.mean() - b.nnz / n_cols) < 1e-9
    assert abs(cdeg.var() - cdeg.mean()) < 0.05 * cdeg.mean()


def test_batch_layout():
    G = 16
    b = gen.batch_mixed(G, n_min=100, n_max=3000, seed=1)
    sizes, degs = gen.batch_plan(G, 100, 3000, seed=1)
    assert b.num_graphs == G and len(b.row_ptr) == b.vtx_off[-1] + G
    for i in range(G):
        g = b.graph(i)
        want = gen.batch_member(i, sizes, degs, seed=1)
        assert g.n == sizes[i]
        assert np.array_equal(g.row_ptr, want.row_ptr) and np.array_equal(g.col_idx, want.col_idx)
        _structure(g, sorted_rows=False)
        if i % 2 == 0:
            assert np.array_equal(g.row_ptr, gen.grid2d(int(sizes[i])).row_ptr)
    assert np.all((sizes >= 100) & (sizes <= 3000))
    assert np.all((degs >= 2) & (degs <= 32))


def test_generators_are_deterministic():
    for f in (lambda: gen.rmat(12, 16, seed=7), lambda: gen.er(5000, 9.0, seed=7),
              lambda: gen.stencil3d(7, 6, 5, points=27), lambda: gen.grid2d(777)):
        a, b = f(), f()
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    x, y = gen.bipartite(5000, 900, seed=3), gen.bipartite(5000, 900, seed=3)
    assert np.array_equal(x.col_idx, y.col_idx) and np.array_equal(x.row_idx, y.row_idx)
    assert not np.array_equal(gen.rmat(12, 16, seed=7).col_idx, gen.rmat(12, 16, seed=8).col_idx)
