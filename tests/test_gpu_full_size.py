"""Parity at full size, in the launch configuration bench.py times.

  * D1 on R-MAT scale 24 (16.8M vertices, ~521M CSR entries);
  * D2 on the 27-point stencil 128^3 (2.1M vertices, 53.6M entries);
  * PD2 on the 4M x 1M random Jacobian pattern (rows 1 + Poisson(7));
  * the batched form on 4096 graphs (half 2D grids, half G(n, m) with
    average degree U[2, 32], sizes log-uniform on [100, 200000]).

The colors are compared with the oracle element by element.  The three
oracle runs take minutes of single-threaded CPU time, so they run in
parallel in spawned worker processes while the GPU side runs here."""
import json
import multiprocessing as mp
import os
import platform
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import oracle
from tests import _full_size_jobs as jobs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oracle_futures():
    ex = ProcessPoolExecutor(max_workers=3, mp_context=mp.get_context("spawn"))
    futs = {k: ex.submit(jobs.oracle_job, k) for k in jobs.CASES}
    yield futs
    ex.shutdown(wait=False, cancel_futures=True)


@pytest.fixture(scope="module")
def batch_oracle_futures():
    import os
    workers = max(1, min(12, (os.cpu_count() or 4) - 3))
    ex = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    idx = list(range(jobs.BATCH_GRAPHS))
    chunks = [idx[k::workers * 4] for k in range(workers * 4)]
    futs = [ex.submit(jobs.batch_oracle_job, c) for c in chunks]
    yield futs
    ex.shutdown(wait=False, cancel_futures=True)


def _record_oracle_time(kind, want):
    """With $PGC_ORACLE_TIMES set, add the oracle's wall time on this
    full-size input (one thread, run beside the others in a worker process)
    to that JSON file: the CPU baseline of the full workload."""
    path = os.environ.get("PGC_ORACLE_TIMES")
    if not path:
        return
    t = want[5]
    d = json.load(open(path)) if os.path.exists(path) else {}
    model = None
    try:
        for l in open("/proc/cpuinfo"):
            if l.lower().startswith(("model name", "cpu part")):
                model = l.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    unit = "entries/s" if kind == "bip_pd2" else "edges/s"
    d[kind] = {"seconds": round(t["seconds"], 2), "value": t["units"] / t["seconds"],
               "unit": unit, "cores": 1, "kind": "oracle", "rounds": int(want[1]),
               "num_colors": int(want[2]), "arch": platform.machine(), "cpu": model,
               "nproc": os.cpu_count(),
               "how": "tests/test_gpu_full_size.py: the oracle on the full input in a spawned "
                      "worker, three such workers in parallel"}
    json.dump(d, open(path, "w"), indent=1)


def _compare(got, rounds, ncol, prof, want):
    w_colors, w_rounds, w_ncol, w_tw, w_ts = want[:5]
    assert rounds == w_rounds and ncol == w_ncol
    diff = np.count_nonzero(got != w_colors)
    assert diff == 0, f"{diff} of {len(got)} colors differ"
    assert np.array_equal(prof.trace_w, w_tw)
    assert np.array_equal(prof.trace_s, w_ts)


def test_rmat24_d1_bit_exact(oracle_futures):
    import torch
    import paper_2107_00075_gb300 as pgc
    g = jobs.make_input("rmat24_d1")
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    prof = pgc.Profile(trace_cap=1 << 16)
    r = pgc.pgc_color_d1(rp, ci, seed=1, profile=prof)
    colors = r.colors.cpu().numpy()
    del rp, ci
    t0 = time.time()
    want = oracle_futures["rmat24_d1"].result()
    print(f"waited {time.time() - t0:.1f} s for the oracle")
    _compare(colors, r.rounds, r.num_colors, prof, want)
    _record_oracle_time("rmat24_d1", want)
    assert oracle.count_improper(oracle.D1, g.row_ptr, g.col_idx, colors) == 0
    assert oracle.count_non_grundy(oracle.D1, g.row_ptr, g.col_idx, colors) == 0


def test_stencil128_d2_bit_exact(oracle_futures):
    import torch
    import paper_2107_00075_gb300 as pgc
    g = jobs.make_input("stencil128_d2")
    assert g.n == 128 ** 3 and g.nnz == 53_645_816
    prof = pgc.Profile(trace_cap=1 << 16)
    r = pgc.pgc_color_d2(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda(),
                         seed=1, profile=prof)
    colors = r.colors.cpu().numpy()
    want = oracle_futures["stencil128_d2"].result()
    _compare(colors, r.rounds, r.num_colors, prof, want)
    _record_oracle_time("stencil128_d2", want)
    assert r.num_colors >= 27


def test_bipartite_pd2_bit_exact(oracle_futures):
    import torch
    import paper_2107_00075_gb300 as pgc
    b = jobs.make_input("bip_pd2")
    assert b.n_rows == 1 << 22 and b.n_cols == 1 << 20
    prof = pgc.Profile(trace_cap=1 << 16)
    t = lambda a: torch.from_numpy(a).cuda()
    r = pgc.pgc_color_pd2(b.n_rows, b.n_cols, t(b.row_ptr), t(b.col_idx), t(b.col_ptr),
                          t(b.row_idx), seed=1, profile=prof)
    colors = r.colors.cpu().numpy()
    want = oracle_futures["bip_pd2"].result()
    _compare(colors, r.rounds, r.num_colors, prof, want)
    _record_oracle_time("bip_pd2", want)
    assert r.num_colors >= np.diff(b.row_ptr).max()


def test_batch4096_bit_exact(batch_oracle_futures):
    import torch
    import paper_2107_00075_gb300 as pgc
    from paper_2107_00075_gb300 import inputs as gen
    b = gen.batch_mixed(jobs.BATCH_GRAPHS)
    t = lambda a: torch.from_numpy(a).cuda()
    r = pgc.pgc_color_d1_batch(t(b.vtx_off), t(b.nnz_off), t(b.row_ptr), t(b.col_idx), seed=1)
    colors = r.colors.cpu().numpy()
    gr = r.rounds_per_graph.cpu().numpy()
    gc = r.colors_per_graph.cpu().numpy()
    seen = 0
    for f in batch_oracle_futures:
        for i, dig, rounds, ncol in f.result():
            a, z = int(b.vtx_off[i]), int(b.vtx_off[i + 1])
            assert jobs.digest(colors[a:z]) == dig, f"graph {i}"
            assert gr[i] == rounds and gc[i] == ncol, f"graph {i}"
            seen += 1
    assert seen == jobs.BATCH_GRAPHS
