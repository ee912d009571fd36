"""The allocation-free entry point, through the C ABI: for callers that may
not have the library allocate device memory, pgc_color_d1_noalloc must give
exactly what pgc_color_d1 gives and what the oracle computes (colors, rounds,
color count), on calls in a row that share its fixed scratch array, and it
must not change the device's free memory.  Collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2107_00075_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


def test_noalloc_matches_pgc_color_d1_and_the_oracle_twice_in_a_row():
    import torch
    import paper_2107_00075_gb300 as pgc
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    graphs = [gen.stencil3d(32, 32, 32, points=7), gen.rmat(13, 16, seed=6)]
    for g, seed, flags in ((graphs[0], 1, 0), (graphs[1], 4, 0), (graphs[1], 4, 0),
                           (graphs[1], 9, pgc.PGC_NO_DEGREE_RULE)):
        rp = torch.from_numpy(g.row_ptr).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        got = pgc.pgc_color_d1_noalloc(rp, ci, seed=seed, colors=out, flags=flags)
        ref = pgc.pgc_color_d1(rp, ci, seed=seed, flags=flags)
        assert got.rounds == ref.rounds and got.num_colors == ref.num_colors
        assert torch.equal(out, ref.colors)
        want = oracle.color_d1(g.row_ptr, g.col_idx, seed=seed,
                               recolor_degrees=not (flags & pgc.PGC_NO_DEGREE_RULE))
        assert got.rounds == want.rounds and got.num_colors == want.num_colors
        assert np.array_equal(out.cpu().numpy(), want.colors)


def test_noalloc_allocates_no_device_memory():
    import torch
    import paper_2107_00075_gb300 as pgc
    g = gen.rmat(12, 16, seed=3)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(3)]
    pgc.pgc_color_d1_noalloc(rp, ci, seed=2, colors=outs[0])   # first call: address lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pgc.pgc_color_d1_noalloc(rp, ci, seed=2, colors=outs[1])
    pgc.pgc_color_d1_noalloc(rp, ci, seed=2, colors=outs[2])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(outs[1], outs[0]) and torch.equal(outs[2], outs[0])


def test_noalloc_rejects_inputs_over_its_limit():
    import torch
    import paper_2107_00075_gb300 as pgc
    g = gen.empty(40000)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_color_d1_noalloc(rp, ci, seed=1, colors=out)
    assert e.value.status == 1 and "32768" in str(e.value)
    with pytest.raises(TypeError):
        pgc.pgc_color_d1_noalloc(g.row_ptr, g.col_idx)
