"""Parity at the benchmark's full size, in the launch configuration bench.py
times: distance-1 coloring of R-MAT scale 24 (16.8M vertices, ~521M CSR
entries) compared with the oracle element by element, plus the properness
and Grundy checks that hold at any size."""
import time

import numpy as np
import pytest

import oracle
from paper_2107_00075_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


def test_rmat24_d1_bit_exact():
    import torch
    import paper_2107_00075_gb300 as pgc
    g = gen.rmat(24, 16, seed=1)
    assert g.n == 1 << 24
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    prof = pgc.Profile(trace_cap=1 << 16)
    r = pgc.pgc_color_d1(rp, ci, seed=1, profile=prof)
    colors = r.colors.cpu().numpy()
    del rp, ci
    t0 = time.time()
    want = oracle.color_d1(g.row_ptr, g.col_idx, seed=1)
    print(f"oracle on R-MAT 24: {time.time() - t0:.1f} s, {want.rounds} rounds")
    assert r.rounds == want.rounds and r.num_colors == want.num_colors
    diff = np.count_nonzero(colors != want.colors)
    assert diff == 0, f"{diff} of {g.n} colors differ"
    assert np.array_equal(prof.trace_w, want.trace_w)
    assert np.array_equal(prof.trace_s, want.trace_s)
    assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, colors) == 0
    assert oracle.count_non_grundy(oracle.D1, g.row_ptr, g.col_idx, colors) == 0
