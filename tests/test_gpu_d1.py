"""GPU parity for distance-1 coloring: the CUDA path through the C ABI must
match the oracle bit for bit (colors, rounds, color count, per-round
worklist sizes) on every input, launch geometry and tier split."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2107_00075_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pgc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2107_00075_gb300 as p
    return p


def dev_csr(g):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(g.row_ptr)).cuda(),
            torch.from_numpy(np.ascontiguousarray(g.col_idx)).cuda())


def run_gpu(pgc, g, seed=1, **kw):
    rp, ci = dev_csr(g)
    prof = pgc.Profile(trace_cap=100000)
    r = pgc.pgc_color_d1(rp, ci, seed=seed, profile=prof, **kw)
    return r.colors.cpu().numpy(), r.rounds, r.num_colors, prof


def assert_parity(pgc, g, seed=1, recolor_degrees=True, **kw):
    flags = kw.pop("flags", 0)
    if not recolor_degrees:
        flags |= pgc.PGC_NO_DEGREE_RULE
    colors, rounds, k, prof = run_gpu(pgc, g, seed=seed, flags=flags, **kw)
    want = oracle.color_d1(g.row_ptr, g.col_idx, seed=seed, recolor_degrees=recolor_degrees)
    assert rounds == want.rounds, (rounds, want.rounds)
    assert k == want.num_colors
    mism = np.nonzero(colors != want.colors)[0]
    assert len(mism) == 0, f"{len(mism)} colors differ, first at {mism[:5]}"
    assert np.array_equal(prof.trace_w, want.trace_w)
    assert np.array_equal(prof.trace_s, want.trace_s)
    return want


def test_worked_examples(pgc):
    cases = json.load(open(os.path.join(GOLDEN, "worked_examples.json")))["cases"]
    for c in cases:
        if c["kind"] != "d1":
            continue
        g = gen.from_edge_list(c["n"], c["edges"])
        flags = 0 if c["recolor_degrees"] else pgc.PGC_NO_DEGREE_RULE
        colors, rounds, k, _ = run_gpu(pgc, g, seed=c["seed"], flags=flags)
        assert list(colors) == c["colors"] and rounds == c["rounds"], c["name"]


@pytest.mark.parametrize("n", [1, 2, 5, 33, 100])
def test_complete_graphs(pgc, n):
    assert_parity(pgc, gen.complete(n), seed=n)


def test_small_random_graphs(pgc):
    for i in range(60):
        g = gen.random_small(3 + i, 0.05 + (i % 7) * 0.1, seed=i)
        assert_parity(pgc, g, seed=i + 1, recolor_degrees=bool(i % 4))


def test_stencil_32cubed(pgc):
    """The 7-point 32^3 stencil (32,768 vertices, 190,464 entries)."""
    g = gen.stencil3d(32, 32, 32, points=7)
    assert g.n == 32768 and g.nnz == 190464
    assert_parity(pgc, g, seed=1)


@pytest.mark.parametrize("mid,hub", [(0, 0), (1, 2), (2, 8), (4, 16), (63, 64), (8, 100000), (1000, 1000)])
def test_rmat_all_tiers(pgc, mid, hub):
    """Skewed degrees with thresholds moved so that every tier (thread,
    warp, block per vertex) carries work, including hubs above 8192 colors'
    worth of degree in the block path."""
    g = gen.rmat(14, 16, seed=3)
    assert_parity(pgc, g, seed=5, mid_degree=mid, hub_degree=hub)


@pytest.mark.parametrize("block,per_sm", [(128, 1), (256, 0), (512, 2), (1024, 1), (256, 7)])
def test_launch_geometry_does_not_change_colors(pgc, block, per_sm):
    g = gen.rmat(13, 8, seed=9)
    assert_parity(pgc, g, seed=2, block=block, grid_per_sm=per_sm, mid_degree=8, hub_degree=64)


def test_host_loop_matches_graph_loop(pgc):
    g = gen.er(20000, 12.0, seed=2)
    assert_parity(pgc, g, seed=3, flags=pgc.PGC_HOST_LOOP)
    assert_parity(pgc, g, seed=3)


def test_host_arrays_are_staged(pgc):
    g = gen.rmat(12, 8, seed=1)
    r = pgc.pgc_color_d1(g.row_ptr, g.col_idx, seed=4)
    want = oracle.color_d1(g.row_ptr, g.col_idx, seed=4)
    assert isinstance(r.colors, np.ndarray)
    assert np.array_equal(r.colors, want.colors) and r.rounds == want.rounds


def test_pinned_host_arrays(pgc):
    """Pinned host arrays (what the end-to-end measurement passes): staged
    on the device, colored, copied back; repeated calls on the same buffers,
    with validation and with the host-driven loop, all equal the oracle."""
    import torch
    g = gen.rmat(14, 16, seed=6)
    rp = torch.from_numpy(g.row_ptr).pin_memory()
    ci = torch.from_numpy(g.col_idx).pin_memory()
    out = torch.empty(g.n, dtype=torch.int32).pin_memory()
    want = oracle.color_d1(g.row_ptr, g.col_idx, seed=8)
    for flags in (0, 0, pgc.PGC_VALIDATE, pgc.PGC_HOST_LOOP):
        r = pgc.pgc_color_d1(rp, ci, seed=8, colors=out, flags=flags)
        assert np.array_equal(out.numpy(), want.colors), flags
        assert r.rounds == want.rounds and r.num_colors == want.num_colors


def test_large_host_arrays_overlapped_upload(pgc):
    """A host adjacency of 2^24 entries or more is uploaded in row ranges
    that overlap the list build; colors and rounds must equal those of the
    same graph given in device memory, from pinned and from pageable host
    memory, with the device loop and with the host-driven loop."""
    import torch
    g = gen.rmat(20, 16, seed=13)
    assert g.nnz >= 1 << 24
    dev = pgc.pgc_color_d1(torch.from_numpy(g.row_ptr).cuda(),
                           torch.from_numpy(g.col_idx).cuda(), seed=2)
    want = dev.colors.cpu().numpy()
    rp = torch.from_numpy(g.row_ptr).pin_memory()
    ci = torch.from_numpy(g.col_idx).pin_memory()
    for args, flags in (((rp, ci), 0), ((rp, ci), 0), ((g.row_ptr, g.col_idx), 0),
                        ((rp, ci), pgc.PGC_HOST_LOOP)):
        r = pgc.pgc_color_d1(*args, seed=2, flags=flags)
        got = r.colors.numpy() if hasattr(r.colors, "numpy") else r.colors
        assert np.array_equal(got, want) and r.rounds == dev.rounds, flags
    assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, want) == 0


def test_edge_cases(pgc):
    import torch
    # n = 0
    r = pgc.pgc_color_d1(torch.zeros(1, dtype=torch.int32, device="cuda"),
                         torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert r.rounds == 0 and r.num_colors == 0
    # edgeless
    for n in (1, 7, 100000):
        assert_parity(pgc, gen.empty(n))
    # self-loops and duplicates
    rp = np.array([0, 3, 5, 6], dtype=np.int32)
    ci = np.array([0, 1, 1, 0, 2, 1], dtype=np.int32)
    from paper_2107_00075_gb300.inputs import CSR
    assert_parity(pgc, CSR(rp, ci))
    # ragged sizes around warp and block multiples
    for n in (31, 32, 33, 255, 256, 257, 1023, 1025):
        assert_parity(pgc, gen.cycle(n), seed=n)


def test_validate_rejects_bad_input(pgc):
    import torch
    rp = torch.tensor([0, 2, 1, 3], dtype=torch.int32, device="cuda")
    ci = torch.tensor([1, 2, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_d1(rp, ci, flags=pgc.PGC_VALIDATE)
    assert e.value.status == 1
    rp = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    ci = torch.tensor([1, 9], dtype=torch.int32, device="cuda")
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_d1(rp, ci, flags=pgc.PGC_VALIDATE)
    assert e.value.status == 1


def test_max_rounds_reports_no_converge(pgc):
    g = gen.complete(20)
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_d1(*dev_csr(g), max_rounds=5)
    assert e.value.status == 4
    # the library stays usable afterwards
    assert_parity(pgc, g)


def test_device_loop_timeout_reports_status(pgc):
    """A 1 ms budget on a coloring that needs far more rounds: the device
    loop stops between rounds with PGC_ERR_TIMEOUT (no hang, no fault)."""
    g = gen.complete(3000)
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_d1(*dev_csr(g), timeout_ms=1)
    assert e.value.status == 5
    assert_parity(pgc, gen.complete(50))


def test_repeatable_and_stream(pgc):
    import torch
    g = gen.rmat(13, 16, seed=4)
    rp, ci = dev_csr(g)
    s = torch.cuda.Stream()
    outs = []
    for _ in range(3):
        with torch.cuda.stream(s):
            outs.append(pgc.pgc_color_d1(rp, ci, seed=8, stream=s).colors.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs)


@pytest.mark.parametrize("tail", [-1, 1, 100, 5000, 1 << 30])
def test_tail_kernel_threshold_does_not_change_colors(pgc, tail):
    """The last rounds run on the subgraph the worklist induces once the
    worklist is small; where the hand-over happens must not change anything."""
    g = gen.rmat(14, 16, seed=11)
    assert_parity(pgc, g, seed=3, tail_vertices=tail)
    assert_parity(pgc, g, seed=3, tail_vertices=tail, flags=pgc.PGC_HOST_LOOP)
    assert_parity(pgc, gen.stencil3d(16, 16, 16, points=7), seed=2, tail_vertices=tail)
