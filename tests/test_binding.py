"""CPU checks of the Python binding: argument marshalling errors are raised
before the library is called, empty problems round-trip, and without a GPU
a real problem fails loudly (there is no CPU fallback)."""
import numpy as np
import pytest

import paper_2107_00075_gb300 as pgc
from paper_2107_00075_gb300 import inputs as gen


def test_type_and_size_errors():
    g = gen.path(5)
    with pytest.raises(TypeError):
        pgc.pgc_color_d1(g.row_ptr.astype(np.int64), g.col_idx)
    with pytest.raises(TypeError):
        pgc.pgc_color_d1(g.row_ptr, np.repeat(g.col_idx, 2)[::2])   # not contiguous
    with pytest.raises(ValueError):
        pgc.pgc_color_d1(g.row_ptr, g.col_idx, colors=np.zeros(3, np.int32))
    with pytest.raises(ValueError):
        pgc.pgc_color_d1(np.zeros(0, np.int32), np.zeros(0, np.int32))
    b = gen.bipartite(20, 10, seed=1)
    with pytest.raises(ValueError):
        pgc.pgc_color_pd2(21, 10, b.row_ptr, b.col_idx, b.col_ptr, b.row_idx)
    with pytest.raises(TypeError):
        pgc.pgc_color_d1_noalloc(g.row_ptr, g.col_idx)            # host arrays refused


def test_empty_problems_round_trip():
    e = gen.empty(0)
    for f in (pgc.pgc_color_d1, pgc.pgc_color_d2):
        prof = pgc.Profile(trace_cap=8)
        r = f(e.row_ptr, e.col_idx, profile=prof)
        assert r.rounds == 0 and r.num_colors == 0 and len(r.colors) == 0
        assert len(prof.trace_w) == 0
    z = np.zeros(1, np.int32)
    r = pgc.pgc_color_pd2(0, 0, z, np.zeros(0, np.int32), z, np.zeros(0, np.int32))
    assert r.rounds == 0 and r.num_colors == 0


def test_option_errors_raise_pgc_error():
    e = gen.empty(0)
    with pytest.raises(pgc.PgcError) as err:
        pgc.pgc_color_d1(e.row_ptr, e.col_idx, block=100)
    assert err.value.status == 1 and "block" in str(err.value)


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = gen.path(10)
    with pytest.raises(pgc.PgcError) as err:
        pgc.pgc_color_d1(g.row_ptr, g.col_idx)
    assert err.value.status == 2          # PGC_ERR_CUDA: no device, no coloring
