"""CPU checks of what bench.py reports: the byte models behind the roofline
(hand-computed on a small trace) and the JSON line of the reference arm."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_design_bytes_on_a_hand_trace():
    # three rounds: |W| = 10, 6, 2; S = 40, 30, 8; H = 20, 12, 4; n = 10, nnz = 40,
    # every degree 4 (no overflow bitmaps, no long rows)
    w, s, h = [10, 6, 2], [40, 30, 8], [20, 12, 4]
    b = bench.d1_algorithmic_bytes(w, s, h, 10, 40, deg=[4] * 10)
    # offsets, degree/color/list-length writes, forbidden word, uncolored
    # bitmap, one 16-byte worklist entry per vertex
    assert b["d1_classify"] == 4 * 11 + 12 * 10 + 8 * 10 + 10 / 8 + 16 * 10
    # entries, adjacency + neighbor degree, kept list entries, list lengths
    assert b["d1_build"] == 16 * 10 + 8 * 40 + 4 * 20 + 4 * 10
    assert b["d1_tier"] == 4 * 10 + 4 * 11 + 16 * 10
    # 16-byte entry, own color, forbidden word, color write; none in round 1
    assert b["d1_assign"] == 32 * 6 + 32 * 2
    # entry + own color per vertex, 8 per list entry (round 1 reads none),
    # 8 per winner, push items (1/16 B per winner adjacency entry), and a
    # 16-byte next-round entry per loser
    won, won_adj, nxt = [4, 4, 2], [10, 22, 8], [6, 2, 0]
    want = sum(20 * a + 8 * l + 8 * x + y / 16 + 16 * z
               for a, l, x, y, z in zip(w, [0, 12, 4], won, won_adj, nxt))
    assert b["d1_detect"] == pytest.approx(want)
    # pushes: adjacency of each round's winners, S_r - S_{r+1}, 16 B each
    assert b["d1_push"] == 16 * (10 + 22 + 8)
    assert "d1_core" not in b


def test_setup_bytes_count_overflow_clears_and_long_rows():
    # one vertex of degree 70 (overflow bitmap of 3 words), one of degree 600
    # (19 words, and two 512-entry build items instead of a worklist entry)
    deg = [70, 600] + [1] * 8
    b = bench.d1_setup_bytes(10, sum(deg), 0, deg)
    clears = 4 * 3 + 4 * 19
    assert b["d1_classify"] == 4 * 11 + 12 * 10 + 8 * 10 + 10 / 8 + 16 * 9 + 8 * 2 + clears
    assert b["d1_build"] == 16 * 9 + 8 * 2 + 8 * sum(deg) + 4 * 10


def test_design_bytes_split_at_the_core_phase():
    w, s, h = [10, 6, 2], [40, 30, 8], [20, 12, 4]
    whole = bench.d1_algorithmic_bytes(w, s, h, 10, 40)
    split = bench.d1_algorithmic_bytes(w, s, h, 10, 40, tail_at=2)
    asg, det, psh = bench.d1_round_bytes(w, s, h)
    assert split["d1_detect"] == pytest.approx(det[0] + det[1])
    # the core phase: extraction (24 B per adjacency entry of W_3) + round 3
    assert split["d1_core"] == pytest.approx(24 * 8 + asg[2] + det[2] + psh[2])
    rounds = lambda d: sum(d[k] for k in ("d1_assign", "d1_detect", "d1_push"))
    assert rounds(split) + split["d1_core"] - 24 * 8 == pytest.approx(rounds(whole))


def test_net_bytes_on_a_hand_trace():
    # two rounds: |W| = 8, 3; nets of W's vertices K = 20, 9; nets visited
    # A = 5 (all) then 4 (marking); their members M = 30, 10
    b = bench.net_algorithmic_bytes([8, 3], [20, 9], [5, 4], [30, 10], 8, 5, 30)
    assert b["net_init"] == 28 * 8 + 12 * 20 + 4 * 5
    assert b["net_assign"] == (16 * 8 + 12 * 20) + (16 * 3 + 12 * 9 + 8 * 9)
    assert b["net_detect"] == (8 * 5 + 12 * 30 + 4 * 3) + (8 * 4 + 4 * 5 + 12 * 10)
    assert b["net_commit"] == (12 * 8 + 16 * 5 + 12 * 11 + 4 * 3) + (12 * 3 + 16 * 3 + 12 * 9)
    assert b["method_detect"] == (8 * 5 + 12 * 30 + 4 * 3) + (8 * 4 + 12 * 10)


def test_roofline_entry_arithmetic(tmp_path, monkeypatch):
    r = bench.roofline_entry("k", 2.0, 4, 8e9, 1000.0, "measured", "net.cu")
    # 2e9 bytes per launch in 0.5 ms = 4000 GB/s
    assert r["alg_bytes_per_launch"] == 2e9 and r["avg_launch_ms"] == 0.5
    assert r["achieved"] == pytest.approx(4000.0) and r["frac"] == pytest.approx(4.0)
    assert r["traffic"] is None and r["dram_frac"] is None


def test_dram_capture_scaling_and_staleness(tmp_path, monkeypatch):
    """traffic and dram_frac come from a committed small capture, looked up by
    workload key, scaled by the design bytes, and dropped once the kernel's
    source file no longer matches the capture's hash."""
    src = tmp_path / "paper_2107_00075_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "net.cu").write_text("kernel v1")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.source_sha("net.cu")
    cap = {"net_detect (d2)": {"workload": "w", "dram_bytes": 3e9, "design_bytes": 6e9,
                               "kernel_source_sha256": sha}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(cap))
    r = bench.roofline_entry("net_detect", 2.0, 4, 8e9, 1000.0, "measured", "net.cu",
                             capture="net_detect (d2)")
    # 2e9 design bytes per launch, half of them from DRAM, in 0.5 ms
    assert r["traffic"] == pytest.approx(1e9) and r["dram_frac"] == pytest.approx(2.0)
    assert r["dram_capture"] == "w"
    other = bench.roofline_entry("net_detect", 2.0, 4, 8e9, 1000.0, "measured", "net.cu",
                                 capture="net_detect (pd2)")
    assert other["traffic"] is None
    (src / "net.cu").write_text("kernel v2")
    stale = bench.roofline_entry("net_detect", 2.0, 4, 8e9, 1000.0, "measured", "net.cu",
                                 capture="net_detect (d2)")
    assert stale["traffic"] is None and stale["dram_frac"] is None


def test_method_bytes_on_a_hand_trace():
    w, s = [10, 6, 2], [40, 30, 8]
    tot, rounds = bench.d1_method_bytes(w, s, 10, 40)
    r1 = 4 * 11 + 8 * 40 + 4 * 10 + 4 * 6
    r2 = 16 * 6 + 8 * 30 + 4 * 2
    r3 = 16 * 2 + 8 * 8 + 4 * 0
    assert rounds == 3 and tot == r1 + r2 + r3
    tot2, rounds2 = bench.d1_method_bytes(w, s, 10, 40, tail_at=1)
    assert rounds2 == 1 and tot2 == r1


def test_reference_arm_json_line():
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--reference-scale", "10"],
                       capture_output=True, text=True, cwd=ROOT, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["warmup"] >= 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
    assert np.isclose(line["e2e"]["value"], line["value"])


def test_summarize_clocks_parses_reasons():
    ts = "2026/12/04 01:02:03.456"
    lines = [f"{ts}, 0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             f"{ts}, 0, 2070, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
             f"{ts}, 0, 1800, 2070, 1300.0, 0x8, Active, Not Active, Not Active, Not Active",
             "garbage line", f"{ts}, 0, [N/A], 2070, 1, 0, a, b, c, d"]
    out = bench.summarize_clocks(lines)
    assert out["samples"] == 3 and out["sm_mhz"] == 1965 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    import datetime
    want = datetime.datetime(2026, 12, 4, 1, 2, 3, 456000).timestamp()
    assert abs(bench.sample_time(lines[0]) - want) < 1e-6
    assert bench.sample_time("garbage line") is None


def _fake_smi(tmp_path, flag, buffered):
    """A stand-in for nvidia-smi: an idle clock normally, a loaded clock with
    sw_power_cap while flag exists; buffered=True holds every line until exit
    (as a block-buffered pipe could), so only the timestamps place them."""
    fake = tmp_path / "fake-smi"
    out = tmp_path / "held.txt"
    emit = f">> {out}" if buffered else ""
    trap = f"trap 'cat {out}; exit 0' TERM\n" if buffered else ""
    fake.write_text(
        "#!/bin/bash\n" + trap +
        "while true; do\n"
        f"  if [ -e {flag} ]; then c=2070; r=Active; else c=345; r='Not Active'; fi\n"
        "  ts=$(date '+%Y/%m/%d %H:%M:%S.%3N')\n"
        f"  echo \"$ts, 0, $c, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, $r\" {emit}\n"
        "  sleep 0.02\n"
        "done\n")
    fake.chmod(0o755)
    return str(fake)


@pytest.mark.parametrize("buffered", [False, True])
def test_clock_sampler_keeps_only_the_timed_region(tmp_path, buffered):
    """Idle samples before and after the timed region must not count."""
    import time
    flag = tmp_path / "loaded"
    s = bench.ClockSampler(0, exe=_fake_smi(tmp_path, flag, buffered))
    s.start()
    s.wait_first(0.5)
    time.sleep(0.2)            # idle samples before the timed region
    flag.write_text("1")
    time.sleep(0.1)
    s.mark()
    time.sleep(0.3)            # the "timed region"
    s.unmark()
    flag.unlink()
    time.sleep(0.2)            # idle samples after it
    out = s.stop()
    assert out["window"] == "timed region" and out["samples"] >= 3
    assert out["sm_mhz"] == 2070 and out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0, exe="/nonexistent/nvidia-smi")
    s.start()
    s.wait_first(0.1)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_serve_plan_and_digest():
    payloads, reqs = bench.serve_plan(50, 8, seed=3)
    assert len(payloads) == 8 and len(reqs) == 50
    assert all(1000 <= n <= 4_000_000 and k in ("d1", "pd2") for k, n, _ in payloads)
    assert [r[0] for r in reqs[:16]] == payloads + payloads     # request j uses payload j mod 8
    assert len({r[1] for r in reqs}) == 50                       # every request its own seed
    assert bench.serve_plan(50, 8, seed=3) == (payloads, reqs)   # deterministic
    d = bench._Digest(100)
    a = np.arange(1, 60, dtype=np.int32)
    b = a.copy()
    b[[3, 7]] = b[[7, 3]]
    assert d(a) == d(a.copy()) and d(a) != d(b)


def test_oracle_job_small_specs():
    secs, units, rounds, ncol = bench.oracle_job(("stencil_d1", 6, 7, 2))
    assert units == 3 * 6 * 6 * 5          # edges of the 7-point stencil 6^3
    assert rounds >= 1 and ncol >= 2 and secs >= 0
    secs, units, rounds, ncol = bench.oracle_job(("bip_pd2", 300, 100))
    assert units > 0 and ncol >= 1
    e = bench.baseline_entry([(2.0, 100.0, 3, 4), (2.0, 300.0, 5, 6)], "edges/s", "x", cores=2)
    assert e["value"] == pytest.approx(400.0 / 2.0) and e["cores"] == 2


def test_d1_split_and_launch_count():
    from types import SimpleNamespace
    prof = SimpleNamespace(trace_w=[100, 60, 30, 9, 4, 1],
                           kernel_ms={"d1_detect": 1.0, "d1_core": 1.0, "d1_assign": 1.0,
                                      "d1_push": 1.0},
                           kernel_launches={"d1_classify": 1, "d1_build": 1, "d1_tier": 1,
                                            "d1_detect": 3, "d1_assign": 2, "d1_push": 3,
                                            "d1_core": 1})
    # rounds 1-3 launch per round, rounds 4.. in the core phase (worklist <= 10)
    assert bench.d1_split(prof, 10) == 3
    assert bench.d1_kernel_launches(prof) == 3 + 3 + 2 + 3 + 4
    prof.kernel_ms.pop("d1_core")
    assert bench.d1_split(prof, 10) is None
