"""bench.py's host logic, without a GPU: the clock record parsing and its
throttle reasons, the issue-limited ALU peak, the LPT split of a job's
events over ranks, the launch count per batch, the reference arm's JSON
line (the oracle's track path on a tiny workload) and the CPU baseline's
bounded, hit-scaled sample."""
import json
import os
import subprocess
import sys
from collections import namedtuple

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_clock_record_gives_median_clock_and_active_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text(
        "0, 2070, 2070, 910.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
        "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    s = bench.ClockSampler(0)
    s.path = str(path)
    s.f = open(path, "a")
    s.proc = subprocess.Popen([sys.executable, "-c", "pass"])
    out = s.stop()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert not path.exists()


def test_clock_sampler_without_nvidia_smi_reports_so():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_alu_peak_is_sms_times_128_lanes_times_clock():
    Props = namedtuple("Props", "multi_processor_count")
    assert bench.alu_peak_ops(Props(152), {"sm_max_mhz": 2070.0}) == 152 * 128 * 2070e6
    assert bench.alu_peak_ops(Props(2), {}) == 2 * 128 * 2070e6


def test_make_events_splits_the_job_over_ranks_once():
    seen = []
    for rank in range(3):
        ids, events = bench.make_events("single_64", 4, 3, rank)
        assert len(events) == len(ids)
        seen += list(ids)
    assert sorted(seen) == list(range(12))
    ids, events = bench.make_events("single_64", 4, 1, 0)
    assert ids == [0, 1, 2, 3] and len(events) == 4


def test_launch_count_per_batch_grows_by_five_per_event():
    assert bench.launches_per_batch(2) - bench.launches_per_batch(1) == 5
    assert bench.launches_per_batch(3, learned=True) == bench.launches_per_batch(3) + 1


def test_reference_arm_prints_one_json_line_of_the_contract():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                        "single_64", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "events/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_cpu_baseline_stops_after_its_budget_and_scales_by_hits(monkeypatch):
    """The oracle runs events in order until the budget has passed; the value
    is the sample's hits per second over the workload's mean hits per event."""
    import time as _time
    import oracle
    Ev = namedtuple("Ev", "n_hits x y z layer")
    events = [Ev(n, None, None, None, None) for n in (1000, 3000, 2000, 6000)]
    clock = {"t": 0.0}
    ran = []

    def fake_run(g, x, y, z, layer, cp=None, cap=None, threads=1):
        ran.append(g)
        clock["t"] += 1.0 if len(ran) < 3 else 4.0   # seconds per event

    monkeypatch.setattr(oracle, "run_event_tracks", fake_run)
    monkeypatch.setattr(bench.synth, "track_geometry", lambda name, n: n)
    monkeypatch.setattr(bench.time, "perf_counter", lambda: clock["t"])
    r = bench.cpu_baseline("stream2000_256", events, budget_s=5.0)
    # 1 s + 1 s + 4 s: the third event crosses the budget, the fourth is not run
    assert ran == [1000, 3000, 2000]
    mean = (1000 + 3000 + 2000 + 6000) / 4
    assert abs(r["value"] - (6000 / 6.0) / mean) < 1e-12
    assert abs(r["sample_events_per_s"] - 3 / 6.0) < 1e-12
    assert r["kind"] == "oracle" and "first 3 events" in r["sample"]
