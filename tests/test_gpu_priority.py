"""GPU parity for the round-varying priorities (PGC_PRIORITY_DYNAMIC,
PGC_PRIORITY_SATURATION; Sec. 3.3, closing paragraph): colors, rounds, color
count and per-round worklist sizes equal the oracle's
(oracle.color_d1_priority) bit for bit; at R-MAT scale 24 the result is a
proper Grundy coloring (the oracle's own full run takes too long there)."""
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


MODES = [(oracle.PRIO_DYNAMIC, "PGC_PRIORITY_DYNAMIC"),
         (oracle.PRIO_SATURATION, "PGC_PRIORITY_SATURATION")]


def check(pgc, g, mode, flag, seed=1, extra=0):
    prof = pgc.Profile(trace_cap=100000)
    r = pgc.pgc_color_d1(dev(g.row_ptr), dev(g.col_idx), seed=seed, profile=prof,
                         flags=getattr(pgc, flag) | extra)
    want = oracle.color_d1_priority(g.row_ptr, g.col_idx, mode, seed=seed)
    got = r.colors.cpu().numpy()
    assert r.rounds == want.rounds and r.num_colors == want.num_colors
    diff = np.nonzero(got != want.colors)[0]
    assert len(diff) == 0, f"{len(diff)} colors differ, first at {diff[:5]}"
    assert np.array_equal(prof.trace_w, want.trace_w)
    assert np.array_equal(prof.trace_s, want.trace_s)


@pytest.mark.parametrize("mode,flag", MODES)
def test_small_graphs(pgc, mode, flag):
    graphs = [gen.from_edge_list(6, [(0, 1), (0, 4), (0, 5), (1, 2), (1, 3), (2, 3), (2, 4)]),
              gen.star(6), gen.complete(40), gen.cycle(257), gen.complete_bipartite(5, 70),
              gen.empty(33), gen.er(5000, 12.0, seed=2), gen.stencil3d(32, 32, 32, points=7)]
    for i, g in enumerate(graphs):
        check(pgc, g, mode, flag, seed=i + 1)


@pytest.mark.parametrize("mode,flag", MODES)
@pytest.mark.parametrize("scale", [12, 16, 18])
def test_rmat(pgc, mode, flag, scale):
    g = gen.rmat(scale, 16, seed=scale)
    check(pgc, g, mode, flag, seed=3)
    if scale == 12:
        check(pgc, g, mode, flag, seed=3, extra=pgc.PGC_HOST_LOOP)


@pytest.mark.parametrize("mode,flag", MODES)
def test_rmat24_proper_and_grundy(pgc, mode, flag):
    g = gen.rmat(24, 16, seed=1)
    r = pgc.pgc_color_d1(dev(g.row_ptr), dev(g.col_idx), seed=1, flags=getattr(pgc, flag))
    c = r.colors.cpu().numpy()
    assert r.num_colors == c.max() and c.min() >= 1
    assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, c) == 0
    assert oracle.count_non_grundy(oracle.D1, g.row_ptr, g.col_idx, c) == 0


def test_batched_equals_single(pgc):
    import torch
    b = gen.batch_mixed(48, n_max=30000, seed=5)
    r = pgc.pgc_color_d1_batch(dev(b.vtx_off), dev(b.nnz_off), dev(b.row_ptr), dev(b.col_idx),
                               seed=2, flags=pgc.PGC_PRIORITY_SATURATION)
    c = r.colors.cpu().numpy()
    for i in range(48):
        g = b.graph(i)
        if g.n == 0:
            continue
        want = oracle.color_d1_priority(g.row_ptr, g.col_idx, oracle.PRIO_SATURATION, seed=2)
        assert np.array_equal(c[b.vtx_off[i]:b.vtx_off[i + 1]], want.colors), f"graph {i}"


def test_flag_combinations_rejected(pgc):
    g = gen.path(5)
    for flags in (pgc.PGC_PRIORITY_DYNAMIC | pgc.PGC_PRIORITY_SATURATION,
                  pgc.PGC_PRIORITY_DYNAMIC | pgc.PGC_NO_DEGREE_RULE,
                  pgc.PGC_PRIORITY_SATURATION | pgc.PGC_ASYNC):
        with pytest.raises(pgc.PgcError) as e:
            pgc.pgc_color_d1(dev(g.row_ptr), dev(g.col_idx), flags=flags)
        assert e.value.status == 1
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_d2(dev(g.row_ptr), dev(g.col_idx), flags=pgc.PGC_PRIORITY_DYNAMIC)
    assert e.value.status == 1
