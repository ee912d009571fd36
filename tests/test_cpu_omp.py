"""The multi-core CPU baseline (OpenMP restatement of the oracle's D1 round
loop) must give the oracle's colors, rounds and color count exactly, for any
thread count: within a round every worklist vertex is independent of the
others (Jacobi first fit, snapshot detection)."""
import shutil

import numpy as np
import pytest

import oracle
from paper_2107_00075_gb300 import inputs as gen

if shutil.which("gcc") is None:
    pytest.skip("gcc not available", allow_module_level=True)
cpu_omp = pytest.importorskip("oracle.cpu_omp")


def _graphs():
    out = [gen.rmat(13, 16, seed=3), gen.rmat(12, 8, seed=9), gen.stencil3d(20, 17, 9, points=7),
           gen.stencil3d(9, 9, 9, points=27), gen.er(3000, 20.0, seed=2), gen.mycielski(8),
           gen.complete(40), gen.star(50), gen.empty(10), gen.empty(0)]
    for i in range(12):
        out.append(gen.random_small(5 + 9 * i, 0.05 + 0.07 * (i % 6), seed=700 + i))
    return out


@pytest.mark.parametrize("threads", [1, 2, 4])
def test_omp_matches_oracle(threads):
    for i, g in enumerate(_graphs()):
        for rd in (True, False):
            want = oracle.color_d1(g.row_ptr, g.col_idx, seed=i + 1, recolor_degrees=rd)
            colors, rounds, k, used = cpu_omp.color_d1(g.row_ptr, g.col_idx, seed=i + 1,
                                                       recolor_degrees=rd, threads=threads)
            assert used == threads
            assert np.array_equal(colors, want.colors), (i, rd)
            assert rounds == want.rounds and k == want.num_colors


def test_omp_self_loops_and_duplicates():
    g = gen.csr_from_edges(6, np.array([0, 0, 1, 2, 3, 3, 4], dtype=np.int32),
                           np.array([0, 1, 2, 2, 4, 4, 5], dtype=np.int32),
                           drop_loops=False, dedup=False)
    want = oracle.color_d1(g.row_ptr, g.col_idx, seed=4)
    colors, rounds, k, _ = cpu_omp.color_d1(g.row_ptr, g.col_idx, seed=4, threads=2)
    assert np.array_equal(colors, want.colors) and rounds == want.rounds


def test_bench_parallel_leg_matches_oracle():
    """bench.py's multi-core CPU leg (a child process) colors the same
    graph as the oracle leg, with the same rounds and color count."""
    import bench
    eps, secs, g, res = bench.oracle_edges_per_s(12)
    assert eps > 0 and g.n == 1 << 12
    for policy in (None, "PASSIVE"):
        par = bench.cpu_parallel_edges_per_s(12, wait_policy=policy)
        assert par is not None and par["nnz"] == g.nnz and par["threads"] >= 1
        assert (par["rounds"], par["num_colors"]) == (res.rounds, res.num_colors)
        assert par["wait_policy"] == (policy or "default")
