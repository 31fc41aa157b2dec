"""bench.py's arithmetic on the host: the metric's algorithmic work, the CPU sample's
scaling, the whole-job value, the peaks and the recorded DRAM traffic.

The metric is algorithmic GMAC/s = N n p (T M + 1) / sweep time. The split-BF16 doubling is
not counted, and neither are the proposals' linear terms. The CPU sample counts the same
work for the particles and steps it ran.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1106_0322_gb300 import synth  # noqa: E402


def _w(name):
    return dict(synth.WORKLOADS[name], name=name)


def test_algorithmic_work_of_the_headline_workload():
    w = _w("hit-region")
    assert bench.algorithmic_gmac(w) == pytest.approx(8192 * 2000 * 200 * (200 * 10 + 1) / 1e9, rel=1e-15)
    # one likelihood evaluation per move plus the initial one, N n p multiply-adds each
    assert bench.algorithmic_gmac(w) == pytest.approx(
        (w["T"] * w["M"] + 1) * w["N"] * w["n"] * w["p"] / 1e9, rel=1e-15)


def test_cpu_sample_counts_the_same_work():
    for name in ("hit-region", "split-large", "paper-18q"):
        w = _w(name)
        assert bench.oracle_gmac(w, w["N"], w["T"]) == pytest.approx(bench.algorithmic_gmac(w), rel=1e-15)
        # a prefix of k steps with N' particles is that share of the work (init included)
        assert bench.oracle_gmac(w, w["N"] // 4, 3) == pytest.approx(
            (w["N"] // 4) * w["n"] * w["p"] * (3 * w["M"] + 1) / 1e9, rel=1e-15)


def test_whole_job_value_is_weak_scaling():
    # 4 ranks, 5 sweeps each of 6.5 GMAC, slowest rank 100 ms: 4 * 5 * 6.5 / 0.1
    assert bench.whole_job_value(6.5, 5, 4, 100.0) == pytest.approx(1300.0)
    assert bench.whole_job_value(6.5, 5, 1, 100.0) * 4 == pytest.approx(bench.whole_job_value(6.5, 5, 4, 100.0))


def test_peaks_come_from_the_measured_file_when_present():
    peaks, src = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert src == "measured"
        assert peaks == json.load(open(path))
    else:
        assert src == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0


def test_recorded_traffic_is_tied_to_the_kernel_source():
    """The committed DRAM bytes per likelihood launch count only while they were captured
    from the current kernel source; they can never be below the launch's algorithmic
    operand bytes (the particle operand A and G, each read once)."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_counters.json")))["hit-region"]
    assert rec["dram_bytes_per_launch"] == rec["dram_read_bytes"] + rec["dram_write_bytes"]
    assert rec["dram_bytes_per_launch"] >= rec["algorithmic_bytes_per_launch"]
    w = synth.WORKLOADS["hit-region"]
    Kp_used = -(-(w["p"] + 1) // 16) * 16  # K rounded to the 16-wide MMA step
    assert rec["algorithmic_bytes_per_launch"] == w["N"] * 2 * Kp_used * 2 + w["n"] * Kp_used * 2
    got = bench.profile_traffic("hit-region")
    if rec["kernel_sha"] == bench.kernel_source_sha():
        assert got == rec["dram_bytes_per_launch"]
    else:
        assert got is None
    assert bench.profile_traffic("no-such-workload") is None


def test_kernel_digest_ignores_comments_only():
    a = "int f(int x) {\n    return x + 1;  // one more\n}\n"
    b = "// the next integer\nint f(int x) {\n    /* plain */ return x + 1;\n\n}\n"
    c = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench.code_digest([a]) == bench.code_digest([b])
    assert bench.code_digest([a]) != bench.code_digest([c])


def test_cli_parses_without_a_gpu():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0
    for flag in ("--gpus", "--steps", "--warmup", "--workload", "--impl"):
        assert flag in out.stdout


def test_isolated_kernel_takes_the_burst_tensor_peak():
    """The likelihood kernel is timed alone (a 200-launch burst at the unthrottled clock), so
    its fraction divides by the burst BF16 peak, not the power-capped sustained one."""
    peak, src = bench.tensor_peak_burst()
    peaks, _ = bench.measured_peaks()
    assert peak == peaks["bf16_tflops"]
    assert "burst" in src
