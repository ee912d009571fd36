"""GPU parity for the batched form: every graph of a batch must get exactly
the colors, round count and color count that the oracle gives for that
graph alone, whatever the batch composition, launch configuration or
autotuner choice."""
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


def mixed_graphs(seed):
    rng = np.random.default_rng(seed)
    gs = [gen.empty(0), gen.empty(1), gen.complete(7), gen.star(40), gen.empty(5)]
    for i in range(40):
        n = int(np.exp(rng.uniform(np.log(2), np.log(3000))))
        k = i % 4
        if k == 0:
            gs.append(gen.grid2d(n))
        elif k == 1:
            gs.append(gen.er(n, float(rng.uniform(2, 32)), seed=seed * 100 + i))
        elif k == 2:
            gs.append(gen.rmat(max(1, int(np.log2(n))), 8, seed=i))
        else:
            gs.append(gen.random_small(min(n, 60), 0.2, seed=i))
    rng.shuffle(gs)
    return gs


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_batch(pgc, b, seed=1, **kw):
    r = pgc.pgc_color_d1_batch(dev(b.vtx_off), dev(b.nnz_off), dev(b.row_ptr), dev(b.col_idx),
                               seed=seed, **kw)
    return (r.colors.cpu().numpy(), r.rounds_per_graph.cpu().numpy(),
            r.colors_per_graph.cpu().numpy(), r.rounds)


def check_against_oracle(b, colors, gr, gc, seed=1, recolor_degrees=True):
    for g in range(b.num_graphs):
        csr = b.graph(g)
        want = oracle.color_d1(csr.row_ptr, csr.col_idx, seed=seed,
                               recolor_degrees=recolor_degrees)
        a, z = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
        assert np.array_equal(colors[a:z], want.colors), f"graph {g}"
        assert gr[g] == want.rounds and gc[g] == want.num_colors, f"graph {g}"


def test_mixed_batch_matches_oracle(pgc):
    b = gen.make_batch(mixed_graphs(1))
    colors, gr, gc, rounds = run_batch(pgc, b, seed=3)
    check_against_oracle(b, colors, gr, gc, seed=3)
    assert rounds == gr.max()


def test_batch_no_degree_rule_and_geometry(pgc):
    b = gen.make_batch(mixed_graphs(2))
    colors, gr, gc, _ = run_batch(pgc, b, seed=5, flags=pgc.PGC_NO_DEGREE_RULE, block=128,
                                  mid_degree=4, hub_degree=16)
    check_against_oracle(b, colors, gr, gc, seed=5, recolor_degrees=False)


@pytest.mark.parametrize("tail", [-1, 1 << 30])
def test_batch_core_phase_hand_over(pgc, tail):
    """The last rounds on the subgraph the worklist induces, with per-graph
    ids, keys and statistics: from round 2 on (a threshold above every
    worklist) or never."""
    b = gen.make_batch(mixed_graphs(4))
    colors, gr, gc, rounds = run_batch(pgc, b, seed=9, tail_vertices=tail)
    check_against_oracle(b, colors, gr, gc, seed=9)
    assert rounds == gr.max()
    colors2, _, _, _ = run_batch(pgc, b, seed=9, tail_vertices=tail, flags=pgc.PGC_HOST_LOOP)
    assert np.array_equal(colors, colors2)


def test_batch_composition_does_not_change_results(pgc):
    gs = mixed_graphs(3)
    b1 = gen.make_batch(gs)
    b2 = gen.make_batch(list(reversed(gs)) + [gen.rmat(12, 16, seed=9)])
    c1, r1, k1, _ = run_batch(pgc, b1, seed=7)
    c2, r2, k2, _ = run_batch(pgc, b2, seed=7)
    G = len(gs)
    for g in range(G):
        h = G - 1 - g
        a1, z1 = int(b1.vtx_off[g]), int(b1.vtx_off[g + 1])
        a2, z2 = int(b2.vtx_off[h]), int(b2.vtx_off[h + 1])
        assert np.array_equal(c1[a1:z1], c2[a2:z2])
        assert r1[g] == r2[h] and k1[g] == k2[h]


def test_batch_equals_single_calls(pgc):
    gs = mixed_graphs(4)[:12]
    b = gen.make_batch(gs)
    colors, gr, gc, _ = run_batch(pgc, b, seed=2)
    for g, csr in enumerate(gs):
        if csr.n == 0:
            assert gr[g] == 0 and gc[g] == 0
            continue
        r = pgc.pgc_color_d1(dev(csr.row_ptr), dev(csr.col_idx), seed=2)
        a, z = int(b.vtx_off[g]), int(b.vtx_off[g + 1])
        assert np.array_equal(colors[a:z], r.colors.cpu().numpy())
        assert gr[g] == r.rounds and gc[g] == r.num_colors


def test_autotune_and_host_arrays(pgc):
    b = gen.batch_mixed(48, n_min=100, n_max=20000, seed=5)
    r = pgc.pgc_color_d1_batch(b.vtx_off, b.nnz_off, b.row_ptr, b.col_idx, seed=1,
                               flags=pgc.PGC_AUTOTUNE)
    check_against_oracle(b, r.colors, r.rounds_per_graph, r.colors_per_graph)
    # second call of the same size class uses the cached choice
    r2 = pgc.pgc_color_d1_batch(b.vtx_off, b.nnz_off, b.row_ptr, b.col_idx, seed=1,
                                flags=pgc.PGC_AUTOTUNE)
    assert np.array_equal(r.colors, r2.colors)


def test_batch_validate_rejects_bad_graph(pgc):
    good = gen.complete(4)
    bad_rp = np.array([0, 1, 3, 2], dtype=np.int32)   # decreasing
    from paper_2107_00075_gb300.inputs import CSR
    b = gen.make_batch([good, CSR(bad_rp, np.array([1, 0, 2], dtype=np.int32))])
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_d1_batch(b.vtx_off, b.nnz_off, b.row_ptr, b.col_idx,
                               flags=pgc.PGC_VALIDATE)
    assert e.value.status == 1
    b = gen.make_batch([good, CSR(np.array([0, 1, 2], np.int32), np.array([1, 5], np.int32))])
    with pytest.raises(pgc.PgcError):
        pgc.pgc_color_d1_batch(b.vtx_off, b.nnz_off, b.row_ptr, b.col_idx,
                               flags=pgc.PGC_VALIDATE)


def test_empty_batches(pgc):
    r = pgc.pgc_color_d1_batch(np.zeros(1, np.int64), np.zeros(1, np.int64),
                               np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert r.rounds == 0
    b = gen.make_batch([gen.empty(0), gen.empty(0)])
    r = pgc.pgc_color_d1_batch(b.vtx_off, b.nnz_off, b.row_ptr, b.col_idx)
    assert list(r.rounds_per_graph) == [0, 0]
