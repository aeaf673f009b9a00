"""Host logic of bench.py, without a GPU: the reference arm's JSON line, the
traffic figure's staleness rule, the clock-sample parser and percentiles."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", "uniform_1e6"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["metric"] == bench.METRIC   # the same metric name as the GPU arm's line
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_workload_configs_cover_every_single_hull_workload():
    from synth import workloads as W
    for name in W.SINGLE:
        kind, n, seed, desc = bench.workload_config(name, None)
        assert n > 0 and desc
        assert bench.workload_config(name, 1234)[1] == 1234


def test_traffic_comes_from_the_committed_profile_while_its_source_is_unchanged():
    import re
    text = open(os.path.join(ROOT, "profiles", "main_filter_normal_1e8.md")).read()
    per_launch = float(re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text).group(1))
    pts = float(re.search(r"points_per_launch:\s*([0-9.eE+]+)", text).group(1))
    src = re.search(r"source_file:\s*(\S+)", text).group(1)
    sha = re.search(r"source_sha:\s*([0-9a-f]+)", text).group(1)
    t = bench.traffic_from_profile("main_filter", "normal_1e8", 100_000_000)
    if bench.source_sha(os.path.join(ROOT, src)) == sha:
        assert t == pytest.approx(per_launch * 1e8 / pts)
        assert bench.traffic_from_profile("main_filter", "normal_1e8", 50_000_000) == pytest.approx(t / 2)
    else:   # the kernel changed since the capture: no traffic figure
        assert t is None
    assert bench.traffic_from_profile("no_such_kernel", "normal_1e8", 1) is None


def test_traffic_is_null_once_the_source_changed(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// kernel\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = bench.source_sha(str(src))
    body = "traffic_bytes_per_launch: 1.5e6\npoints_per_launch: 1e6\nsource_file: k.cu\nsource_sha: {}\n"
    (prof / "kern_w.md").write_text(body.format(sha))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profile("kern", "w", 2_000_000) == pytest.approx(3.0e6)
    src.write_text("// kernel, changed\n")
    assert bench.traffic_from_profile("kern", "w", 2_000_000) is None


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_median_and_reasons():
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.lines = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1250.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi():
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_percentiles():
    xs = list(range(1, 101))
    assert bench._pct(xs, 50) == 51 or bench._pct(xs, 50) == 50
    assert bench._pct(xs, 99) == 99
    assert bench._pct([], 50) is None
    assert bench._pct([7.0], 99) == 7.0


def test_roofline_entry_arithmetic():
    r = bench.roofline_entry("main_filter", 800e6, 137.5e-6, 6682.5, "measured", 810.3e6)
    assert r["achieved"] == pytest.approx(800e6 / 137.5e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6682.5)
    assert r["frac_of_nominal"] == pytest.approx(r["achieved"] / 7900.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 810.3e6
    assert r["avg_launch_ms"] == pytest.approx(0.1375)


def test_cpu_baseline_and_comparator_legs():
    """The CPU-baseline leg's two parts run on the host alone: the oracle on
    one core, and the multi-core comparator on one thread and on every core."""
    base = bench.cpu_baseline("normal", 1, 0.05)
    assert base["kind"] == "oracle" and base["cores"] == 1 and base["value"] > 0
    hh = bench.cpu_heaphull("normal", 1, 0.05)
    assert hh["cores"] == (os.cpu_count() or 1)
    assert hh["value_1_thread"] > 0 and hh["value_all_cores"] > 0


def test_algorithmic_bytes_follow_the_counters():
    sparse = {"raw": 1000, "records": 900, "two_pass": 0, "stage": 0}
    a = bench.algorithmic_bytes(10_000, sparse)
    assert a == {"main_filter": 8 * 10_000 + 12 * 1000, "post": 12 * 1000 + 12 * 900}
    dense = {"raw": 70_000, "records": 9_000, "two_pass": 1, "stage": 1}
    b = bench.algorithmic_bytes(10_000, dense)
    assert b["post"] == 8 * 10_000 + 12 * 9_000
    assert b["bk_part1"] == b["bk_part2"] == 24 * 9_000 and b["bk_hist"] == 4 * 9_000 and b["bk_hull"] == 12 * 9_000


def test_kernel_rooflines_pick_the_slowest_kernel_with_bytes():
    prof = {"main_filter": (10, 1.0), "post": (10, 3.0), "hull_chains": (10, 9.0)}
    algo = {"main_filter": 8e6, "post": 2e6}
    per, roof = bench.kernel_rooflines(prof, algo, 1000.0, "measured", "nowhere", 1_000_000)
    assert roof["kernel"] == "post"   # hull_chains has no byte count
    assert roof["achieved"] == pytest.approx(2e6 / 0.3e-3 / 1e9)
    assert per["main_filter"]["achieved_gbs"] == pytest.approx(8e6 / 0.1e-3 / 1e9)
    assert roof["traffic"] is None


def test_batch_trace_summary():
    """The server trace (8 values per batch, as ch_server_trace writes them)
    reduced to percentiles and the slowest 1 % of the batches."""
    assert bench.batch_trace_summary([]) is None
    rows = []
    for i in range(200):   # batch i: i % 10 + 1 requests, host time i ms, one set redone every 50
        rows.append((float(i), float(i % 10 + 1), 1000.0 * (i + 1), 0.5, 0.25, 0.1, float(i), float(i % 50 == 0)))
    s = bench.batch_trace_summary(rows)
    assert s["batches"] == 200 and s["sets_redone"] == 4
    assert s["copy_in_ms_p50"] == pytest.approx(0.5) and s["hull_ms_p99"] == pytest.approx(0.25)
    assert s["host_ms_p50"] == pytest.approx(99.5) and s["requests_p99"] == pytest.approx(10.0)
    # the slowest 1 %: host time at or above its 99th percentile (197.01 ms): batches 198 and 199
    assert s["slowest_1pct_mean"]["host_ms"] == pytest.approx(198.5)
    assert s["slowest_1pct_mean"]["points"] == pytest.approx(1000.0 * 199.5)
