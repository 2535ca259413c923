"""Host logic of bench.py without a GPU: the clock record that rejects a
timed run (samples inside the timed window, the median SM clock, throttle
reasons) from synthetic nvidia-smi lines, and the bookkeeping of stored ncu
figures (fingerprints of the captured sources, utilisation weights)."""
import datetime
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _line(t, mhz, reasons=("Not Active",) * 4, max_mhz=2032):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, "0", str(mhz), str(max_mhz), "900.0", "0x0", *reasons])


def _sampler(lines, t0, t1):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    s.t0, s.t1 = t0, t1
    return s


def test_samples_inside_the_window_give_median_clock_and_reasons():
    t0 = 1_700_000_000.0
    lines = [_line(t0 - 5, 345)]                              # idle, before the window
    lines += [_line(t0 + 0.1 * i, mhz) for i, mhz in enumerate([2032, 2010, 2032, 1995, 2032])]
    lines += [_line(t0 + 0.25, 2032, ("Not Active", "Not Active", "Not Active", "Active"))]
    lines += [_line(t0 + 9, 345, ("Active", "Not Active", "Not Active", "Not Active"))]   # after the window
    lines += ["garbage", "2024/01/01, short"]
    s = _sampler(lines, t0, t0 + 0.5).summary()
    assert s["samples"] == 6 and s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"] and s["nearest_outside_window"] is False
    assert abs(s["window_s"] - 0.5) < 1e-9


def test_a_window_shorter_than_the_sampling_period_uses_the_nearest_samples():
    t0 = 1_700_000_000.0
    lines = [_line(t0 - 1.0, 2032), _line(t0 + 0.3, 1900, ("Not Active", "Active", "Not Active", "Not Active")),
             _line(t0 + 2.0, 2032), _line(t0 + 5.0, 345)]
    s = _sampler(lines, t0 + 0.05, t0 + 0.06).summary()
    assert s["nearest_outside_window"] is True and s["samples"] == 3
    assert "hw_thermal_slowdown" in s["reasons"]


def test_no_samples_at_all():
    s = _sampler([], 1.0, 2.0).summary()
    assert s["sm_mhz"] is None and s["samples"] == 0 and s["reasons"] == []


def _run_bench(args, env_extra=None, timeout=300):
    import json
    import subprocess
    env = dict(os.environ)
    env.update(env_extra or {})
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], cwd=root, env=env,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the oracle on the host (no GPU): one
    JSON line with the metric, its own e2e and cpu_baseline, the sample
    sized from the time budget."""
    out = _run_bench(["--impl", "reference", "--steps", "3", "--warmup", "3", "--ref-total-seconds", "3"])
    assert len(out) == 1
    d = out[0]
    assert d["impl"] == "reference" and d["metric"] == "model-count throughput at n=36 (Gassign/s)"
    assert d["unit"] == "Gassign/s" and d["higher_is_better"] is True and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["cores"] >= 1
    assert "2^" in d["cpu_baseline"]["sample"]


def test_reference_arm_other_ranks_exit_quietly():
    out = _run_bench(["--impl", "reference", "--steps", "3", "--warmup", "3", "--ref-total-seconds", "2"],
                     {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out == []


def test_ncu_figures_are_reported_only_for_the_captured_sources():
    """A stored ncu figure carries the fingerprint of the kernel sources it was
    captured on; for any other build the bench reports null and the reason."""
    table = {"sources_sha": "abc", "traffic_step": 7, "vector_lop3_step": 9}
    fresh = bench.ncu_figures(table, "abc", ["traffic_step", "vector_lop3_step"])
    assert fresh == {"traffic_step": 7, "vector_lop3_step": 9, "stale": False}
    stale = bench.ncu_figures(table, "def", ["traffic_step"])
    assert stale["traffic_step"] is None and stale["stale"] and "abc" in stale["reason"] and "def" in stale["reason"]
    none = bench.ncu_figures({}, "def", ["traffic_step"])
    assert none["traffic_step"] is None and none["reason"] == "no capture recorded"


def test_kernel_fingerprint_follows_sources_and_shapes():
    """The fingerprint is a function of the generated kernel sources: equal
    for the same text and shape, different when a shape option changes."""
    import paper_1310_6978_b300 as F
    from paper_1310_6978_b300 import _lib as L
    from paper_1310_6978_b300 import workloads as W
    a = F.compile(W.TRANSITIVE6.text, W.TRANSITIVE6.k)
    b = F.compile(W.TRANSITIVE6.text, W.TRANSITIVE6.k)
    assert bench.kernel_fingerprint([a], 0) == bench.kernel_fingerprint([b], 0)
    b.set_option(L.OPT_REGS_LOG2, 3)
    assert bench.kernel_fingerprint([a], 0) != bench.kernel_fingerprint([b], 0)
    assert bench.kernel_fingerprint([a], 0) != bench.kernel_fingerprint([a], 1)


def test_ncu_utilisation_weights_launches_by_active_cycles():
    per = {"issue_slots_used_pct": [40.0, 60.0, 10.0], "alu_pipe_pct": [70.0, 80.0, 30.0],
           "sm_active_cycles": [100, 300, 0], "sm_elapsed_cycles": [200, 300, 50]}
    u = bench.ncu_utilisation(per)
    assert abs(u["issue_slots_used_pct_weighted"] - 55.0) < 1e-12
    assert abs(u["alu_pipe_pct_weighted"] - 77.5) < 1e-12
    assert u["sm_active_share"] == [0.5, 1.0, 0.0]
    stored = bench.ncu_utilisation(bench.NCU_COUNT["per_launch"])
    assert 0 < stored["issue_slots_used_pct_weighted"] <= 100 and 0 < stored["alu_pipe_pct_weighted"] <= 100
