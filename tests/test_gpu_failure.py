"""Failure paths on the GPU, reached without faulting anything:

  * the core loop's grid barrier gives up (one block held back by a bounded,
    host-set delay; a short poll limit) and the call returns PGC_ERR_TIMEOUT
    with the context usable;
  * an injected allocation failure returns PGC_ERR_OOM, leaves no scratch
    behind, and the next call succeeds;
  * PGC_VALIDATE rejects a non-symmetric graph (D1, D2) and a CSC that does
    not describe the CSR's pattern (PD2) before any coloring work.

Every wait in the library is bounded, so none of these can hang."""
import numpy as np
import pytest

import oracle
from paper_2107_00075_gb300 import inputs as gen
from tests import _graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pgc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2107_00075_gb300 as p
    yield p
    p.pgc_test_core_barrier(0, -1, 0)
    p.pgc_test_fail_alloc(-1)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def d1_matches_oracle(pgc, g, seed=1):
    r = pgc.pgc_color_d1(dev(g.row_ptr), dev(g.col_idx), seed=seed)
    want = oracle.color_d1(g.row_ptr, g.col_idx, seed=seed)
    assert r.rounds == want.rounds and r.num_colors == want.num_colors
    assert np.array_equal(r.colors.cpu().numpy(), want.colors)


@pytest.mark.parametrize("host_loop", [False, True])
def test_core_barrier_gives_up_and_library_recovers(pgc, host_loop):
    # K_64: after round 1 the worklist (63 vertices) is below the core-phase
    # threshold, so the remaining rounds run in the cooperative core loop
    g = gen.complete(64)
    flags = pgc.PGC_HOST_LOOP if host_loop else 0
    pgc.pgc_test_core_barrier(polls=200, slow_block=1, slow_us=50_000)
    try:
        with pytest.raises(pgc.PgcError) as e:
            pgc.pgc_color_d1(dev(g.row_ptr), dev(g.col_idx), seed=3, flags=flags)
        assert e.value.status == 5 and "grid barrier" in str(e.value)
    finally:
        pgc.pgc_test_core_barrier(0, -1, 0)
    d1_matches_oracle(pgc, g, seed=3)
    d1_matches_oracle(pgc, gen.rmat(12, 16, seed=2), seed=5)


def test_late_block_within_the_poll_limit_changes_nothing(pgc):
    # the same late block with the default poll limit (about a second): the
    # barrier simply waits, and the colors are the oracle's
    g = gen.complete(40)
    pgc.pgc_test_core_barrier(0, slow_block=1, slow_us=2_000)
    try:
        d1_matches_oracle(pgc, g, seed=9)
    finally:
        pgc.pgc_test_core_barrier(0, -1, 0)


@pytest.mark.parametrize("after", [0, 3, 6])
def test_injected_oom_releases_scratch(pgc, after):
    import torch
    g = gen.rmat(14, 16, seed=3)
    rp, ci = dev(g.row_ptr), dev(g.col_idx)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pgc.pgc_color_d1(rp, ci, seed=1, colors=out)
    pgc.pgc_release()
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    pgc.pgc_test_fail_alloc(after)
    try:
        with pytest.raises(pgc.PgcError) as e:
            pgc.pgc_color_d1(rp, ci, seed=1, colors=out)
        assert e.value.status == 3 and "injected" in str(e.value)
    finally:
        pgc.pgc_test_fail_alloc(-1)
    torch.cuda.synchronize()
    # the failed call keeps none of the scratch it had grown (allocation
    # granularity of the driver: a few MB of slack)
    assert torch.cuda.mem_get_info()[0] >= free_before - (8 << 20)
    d1_matches_oracle(pgc, g, seed=1)


def test_injected_oom_in_distance2(pgc):
    g = gen.stencil3d(10, 9, 8, points=27)
    pgc.pgc_test_fail_alloc(1)
    try:
        with pytest.raises(pgc.PgcError) as e:
            pgc.pgc_color_d2(dev(g.row_ptr), dev(g.col_idx), seed=2)
        assert e.value.status == 3
    finally:
        pgc.pgc_test_fail_alloc(-1)
    r = pgc.pgc_color_d2(dev(g.row_ptr), dev(g.col_idx), seed=2)
    want = oracle.color_d2(g.row_ptr, g.col_idx, seed=2)
    assert np.array_equal(r.colors.cpu().numpy(), want.colors)


def _drop_one_direction(g):
    """g without the entry (v, u) of its first edge with v < u (u keeps v)."""
    rp, ci = g.row_ptr.copy(), g.col_idx.copy()
    for v in range(g.n):
        row = ci[rp[v]:rp[v + 1]]
        k = np.nonzero(row > v)[0]
        if len(k):
            e = rp[v] + k[0]
            ci = np.delete(ci, e)
            rp[v + 1:] -= 1
            return rp, ci
    raise AssertionError("no edge")


@pytest.mark.parametrize("sorted_rows", [True, False])
def test_validate_rejects_nonsymmetric_graph(pgc, sorted_rows):
    g = gen.rmat(10, 8, seed=7)
    rp, ci = _drop_one_direction(g)
    if not sorted_rows:   # reverse every row: the exact lookup is skipped,
        for v in range(g.n):   # the multiset test still sees the mismatch
            ci[rp[v]:rp[v + 1]] = ci[rp[v]:rp[v + 1]][::-1].copy()
    for f in (pgc.pgc_color_d1, pgc.pgc_color_d2):
        with pytest.raises(pgc.PgcError) as e:
            f(dev(rp), dev(ci), seed=1, flags=pgc.PGC_VALIDATE)
        assert e.value.status == 1 and "symmetric" in str(e.value)
    # the untouched graph passes, with unsorted rows too
    for f in (pgc.pgc_color_d1, pgc.pgc_color_d2):
        f(dev(g.row_ptr), dev(g.col_idx), seed=1, flags=pgc.PGC_VALIDATE)
    ci2 = g.col_idx.copy()
    for v in range(g.n):
        ci2[g.row_ptr[v]:g.row_ptr[v + 1]] = ci2[g.row_ptr[v]:g.row_ptr[v + 1]][::-1].copy()
    r = pgc.pgc_color_d1(dev(g.row_ptr), dev(ci2), seed=1, flags=pgc.PGC_VALIDATE)
    assert r.num_colors > 0


def test_validate_rejects_inconsistent_csc(pgc):
    b = gen.bipartite(300, 120, seed=4)
    args = [dev(x) for x in (b.row_ptr, b.col_idx, b.col_ptr, b.row_idx)]
    pgc.pgc_color_pd2(b.n_rows, b.n_cols, *args, seed=1, flags=pgc.PGC_VALIDATE)
    # move one CSC entry to another row of the same column: same shapes and
    # counts, a different pattern
    ri = b.row_idx.copy()
    c = int(np.argmax(np.diff(b.col_ptr) > 0))
    ri[b.col_ptr[c]] = (ri[b.col_ptr[c]] + 1) % b.n_rows
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_pd2(b.n_rows, b.n_cols, args[0], args[1], args[2], dev(ri), seed=1,
                          flags=pgc.PGC_VALIDATE)
    assert e.value.status == 1 and "same pattern" in str(e.value)
    # an id out of range in the CSC
    ri = b.row_idx.copy()
    ri[0] = b.n_rows + 5
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_pd2(b.n_rows, b.n_cols, args[0], args[1], args[2], dev(ri), seed=1,
                          flags=pgc.PGC_VALIDATE)
    assert e.value.status == 1 and "out of range" in str(e.value)
    # a valid pattern from hand-written rows
    h = _graphs.bipartite_from_rows([[0, 2], [1, 2], [0, 1, 3]], 4)
    r = pgc.pgc_color_pd2(h.n_rows, h.n_cols, *[dev(x) for x in (h.row_ptr, h.col_idx,
                                                                  h.col_ptr, h.row_idx)],
                          seed=1, flags=pgc.PGC_VALIDATE)
    assert r.num_colors == 3
