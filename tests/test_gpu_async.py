"""GPU checks of the asynchronous speculation mode (PGC_ASYNC, Sec. 3.2: the
first fit also avoids tentative colors written in the same round, as
KokkosKernels' in-place VB_BIT does).  Its result depends on timing, so it is
checked by what every such result must satisfy, on every D1 configuration:
a proper coloring (no equal colors across an edge, every vertex colored),
every color at most deg(v) + 1 (first fit over at most deg(v) colors),
rounds at most n, num_colors = the largest color, and the per-round
worklist sizes strictly decreasing."""
import numpy as np
import pytest

import oracle
from paper_2107_00075_gb300 import inputs as gen

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


def check_async(pgc, g, seed=1, flags=0, full_check=True):
    prof = pgc.Profile(trace_cap=1 << 14)
    r = pgc.pgc_color_d1(dev(g.row_ptr), dev(g.col_idx), seed=seed, profile=prof,
                         flags=flags | pgc.PGC_ASYNC)
    c = r.colors.cpu().numpy()
    deg = np.diff(g.row_ptr)
    assert c.min() >= 1 and r.num_colors == c.max()
    assert np.all(c <= deg + 1)
    assert 1 <= r.rounds <= g.n
    tw = prof.trace_w
    assert tw[0] == g.n and all(a > b for a, b in zip(tw, tw[1:]))
    if full_check:
        assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, c) == 0
    return r


@pytest.mark.parametrize("degree_rule", [True, False])
def test_small_graphs(pgc, degree_rule):
    flags = 0 if degree_rule else pgc.PGC_NO_DEGREE_RULE
    for g in (gen.complete(30), gen.star(50), gen.cycle(101), gen.path(2),
              gen.complete_bipartite(7, 9), gen.empty(10), gen.er(3000, 12.0, seed=3),
              gen.stencil3d(17, 9, 5, points=27)):
        check_async(pgc, g, seed=4, flags=flags)


def test_stencil_32cubed_and_rmat(pgc):
    check_async(pgc, gen.stencil3d(32, 32, 32, points=7))
    for seed in (1, 2):
        check_async(pgc, gen.rmat(14, 16, seed=seed), seed=seed)
        check_async(pgc, gen.rmat(14, 16, seed=seed), seed=seed, flags=pgc.PGC_HOST_LOOP)


def test_rmat24_full_size(pgc):
    g = gen.rmat(24, 16, seed=1)
    r = check_async(pgc, g, full_check=False)
    c = r.colors.cpu().numpy()
    # properness over all 520M entries: every edge's endpoints differ
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    assert not np.any(c[rows] == c[g.col_idx]), "adjacent vertices share a color"


def test_batched(pgc):
    import torch
    b = gen.batch_mixed(64, n_max=20000, seed=3)
    r = pgc.pgc_color_d1_batch(dev(b.vtx_off), dev(b.nnz_off), dev(b.row_ptr), dev(b.col_idx),
                               seed=1, flags=pgc.PGC_ASYNC)
    c = r.colors.cpu().numpy()
    for i in range(64):
        g = b.graph(i)
        ci = c[b.vtx_off[i]:b.vtx_off[i + 1]]
        if g.n == 0:
            continue
        assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, ci) == 0
        assert np.all(ci <= np.diff(g.row_ptr) + 1)
