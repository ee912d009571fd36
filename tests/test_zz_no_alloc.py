"""The allocation-free entry point, through the C ABI: for callers that may
not have the library allocate device memory, pgc_color_d1_noalloc must give
exactly what pgc_color_d1 gives (colors, rounds, color count), on two calls
in a row that share its fixed scratch array.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2107_00075_gb300 import inputs as gen

pytestmark = pytest.mark.gpu


def _noalloc(L, rp, ci, n, seed, out, flags=0):
    import torch
    rounds, ncol = ctypes.c_int32(0), ctypes.c_int32(0)
    st = L.pgc_color_d1_noalloc(n, ctypes.c_void_p(rp.data_ptr()),
                                ctypes.c_void_p(ci.data_ptr() if ci.numel() else 0),
                                ctypes.c_uint64(seed), ctypes.c_void_p(out.data_ptr()),
                                ctypes.byref(rounds), ctypes.byref(ncol), ctypes.c_uint32(flags),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, rounds.value, ncol.value


def test_noalloc_matches_pgc_color_d1_twice_in_a_row():
    import torch
    import paper_2107_00075_gb300 as pgc
    from paper_2107_00075_gb300 import binding
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    L = binding.lib()
    L.pgc_color_d1_noalloc.restype = ctypes.c_int
    graphs = [gen.stencil3d(32, 32, 32, points=7), gen.rmat(13, 16, seed=6)]
    for g, seed, flags in ((graphs[0], 1, 0), (graphs[1], 4, 0), (graphs[1], 4, 0),
                           (graphs[1], 9, pgc.PGC_NO_DEGREE_RULE)):
        rp = torch.from_numpy(g.row_ptr).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        st, rounds, ncol = _noalloc(L, rp, ci, g.n, seed, out, flags)
        assert st == 0, L.pgc_last_error()
        ref = pgc.pgc_color_d1(rp, ci, seed=seed, flags=flags)
        assert rounds == ref.rounds and ncol == ref.num_colors
        assert torch.equal(out, ref.colors)


def test_noalloc_rejects_inputs_over_its_limit():
    import torch
    from paper_2107_00075_gb300 import binding
    L = binding.lib()
    L.pgc_color_d1_noalloc.restype = ctypes.c_int
    g = gen.empty(40000)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    st, _, _ = _noalloc(L, rp, ci, g.n, 1, out)
    assert st == 1 and b"32768" in L.pgc_last_error()
