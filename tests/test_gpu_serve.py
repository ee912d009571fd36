"""GPU tests of the served form: requests submitted concurrently from several
threads, admitted by HBM footprint, running overlapped on the device; every
result must equal the same request colored alone."""
import threading

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


def make_requests(count, seed, n_min=1000, n_max=60000):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        if rng.random() < 0.7:
            scale = int(np.ceil(np.log2(n)))
            g = gen.rmat(scale, 8, seed=seed * 7919 + i, n_vertices=n)
            reqs.append(("d1", g, int(rng.integers(1, 1 << 40))))
        else:
            b = gen.bipartite(max(1, int(0.8 * n)), max(1, int(0.2 * n)), seed=seed * 31 + i)
            reqs.append(("pd2", b, int(rng.integers(1, 1 << 40))))
    return reqs


def alone(pgc, kind, x, seed):
    if kind == "d1":
        r = pgc.pgc_color_d1(x.row_ptr, x.col_idx, seed=seed)
    else:
        r = pgc.pgc_color_pd2(x.n_rows, x.n_cols, x.row_ptr, x.col_idx, x.col_ptr, x.row_idx,
                              seed=seed)
    return r.colors, r.rounds, r.num_colors


def submit(srv, kind, x, seed):
    if kind == "d1":
        return srv.submit_d1(x.row_ptr, x.col_idx, seed=seed)
    return srv.submit_pd2(x.n_rows, x.n_cols, x.row_ptr, x.col_idx, x.col_ptr, x.row_idx,
                          seed=seed)


def test_mixed_requests_equal_alone(pgc):
    reqs = make_requests(36, seed=1)
    ids = [None] * len(reqs)
    with pgc.PgcServer(hbm_budget_bytes=1 << 30, max_active=8) as srv:
        def producer(k):
            for i in range(k, len(reqs), 4):
                kind, x, seed = reqs[i]
                ids[i] = submit(srv, kind, x, seed)
        ts = [threading.Thread(target=producer, args=(k,)) for k in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        results = [srv.wait(rid) for rid in ids]
        stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["peak_bytes"] <= stats["budget_bytes"]
    assert stats["max_active_seen"] > 1, "requests never overlapped"
    for (kind, x, seed), (colors, info) in zip(reqs, results):
        want, rounds, ncol = alone(pgc, kind, x, seed)
        assert np.array_equal(colors, want), kind
        assert info.rounds == rounds and info.num_colors == ncol
        assert info.t_submit_ns <= info.t_admit_ns <= info.t_done_ns


def test_small_requests_match_oracle(pgc):
    reqs = make_requests(10, seed=2, n_min=200, n_max=3000)
    with pgc.PgcServer(hbm_budget_bytes=256 << 20, max_active=4) as srv:
        ids = [submit(srv, *r) for r in reqs]
        out = [srv.wait(i) for i in ids]
    for (kind, x, seed), (colors, info) in zip(reqs, out):
        if kind == "d1":
            w = oracle.color_d1(x.row_ptr, x.col_idx, seed=seed)
        else:
            w = oracle.color_pd2(x.n_rows, x.n_cols, x.row_ptr, x.col_idx, x.col_ptr,
                                 x.row_idx, seed=seed)
        assert np.array_equal(colors, w.colors) and info.rounds == w.rounds


def test_admission_by_footprint(pgc):
    """A budget that fits one large request at a time: they run one after
    another, the arena never exceeds the budget, and all finish correctly."""
    g = gen.rmat(16, 8, seed=3)
    with pgc.PgcServer(hbm_budget_bytes=1 << 30, max_active=4) as srv:
        rid = srv.submit_d1(g.row_ptr, g.col_idx)
        _, info = srv.wait(rid)
        fp = info.footprint_bytes
    budget = int(fp * 1.5)
    with pgc.PgcServer(hbm_budget_bytes=budget, max_active=4) as srv:
        ids = [srv.submit_d1(g.row_ptr, g.col_idx, seed=s) for s in (1, 2, 3)]
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["max_active_seen"] == 1 and st["peak_bytes"] <= budget
    for s, (colors, info) in zip((1, 2, 3), res):
        assert np.array_equal(colors, alone(pgc, "d1", g, s)[0])
    # a request larger than the whole budget is refused at submit
    with pgc.PgcServer(hbm_budget_bytes=1 << 20, max_active=2) as srv:
        with pytest.raises(pgc.PgcError) as e:
            srv.submit_d1(g.row_ptr, g.col_idx)
        assert e.value.status == 6
        assert srv.stats()["rejected"] == 1


def test_poll_timeout_unknown_and_device_outputs(pgc):
    import torch
    g = gen.rmat(15, 8, seed=4)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pgc.PgcServer(hbm_budget_bytes=512 << 20, max_active=2) as srv:
        rid = srv.submit_d1(g.row_ptr, g.col_idx, seed=5, colors=out)
        res = None
        while res is None:
            res = srv.poll(rid)
        with pytest.raises(pgc.PgcError) as e:
            srv.wait(rid)
        assert e.value.status == 7
    assert torch.equal(out.cpu(), torch.from_numpy(alone(pgc, "d1", g, 5)[0]))


def test_pd2_needing_more_than_128_colors_is_retried(pgc):
    """A PD2 request whose coloring needs more colors than the first mask
    size is re-run transparently with larger masks."""
    from tests import _graphs
    rows = [list(range(200))] + [[i, (i + 7) % 200] for i in range(50)]
    b = _graphs.bipartite_from_rows(rows, 200)
    with pgc.PgcServer(hbm_budget_bytes=64 << 20, max_active=2) as srv:
        rid = srv.submit_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                             seed=3)
        colors, info = srv.wait(rid)
    want = oracle.color_pd2(b.n_rows, b.n_cols, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx,
                            seed=3)
    assert info.num_colors == 200 and np.array_equal(colors, want.colors)
