"""Host-side logic of bench.py on CPU: the clock sampler's parsing and time window, the launch
count per training step, and the algorithmic byte counts."""
import datetime
import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(lines):
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    c = bench.ClockSampler(0)
    c.proc, c.path = _Done(), path
    return c


def _row(t, sm, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, "0", str(sm), "2070", "900.5", "0x0000000000000000", *reasons])


def test_clock_sampler_keeps_the_samples_of_the_timed_region():
    t0 = 1_800_000_000.0
    lines = [_row(t0 - 0.4, 1200), _row(t0 + 0.01, 2070), _row(t0 + 0.06, 2055), _row(t0 + 0.11, 2070),
             _row(t0 + 0.5, 900), "garbage line"]
    got = _sampler_with(lines).stop(t0, t0 + 0.12)
    assert got["samples"] == 3 and got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == []


def test_clock_sampler_reports_throttle_reasons_and_falls_back_to_all_samples():
    t0 = 1_800_000_000.0
    hot = ("Active", "Not Active", "Not Active", "Active")  # hw_slowdown, sw_power_cap
    lines = [_row(t0, 1800, hot), _row(t0 + 0.05, 1900)]
    got = _sampler_with(lines).stop(t0 + 10.0, t0 + 11.0)  # no sample inside: every sample counts
    assert got["samples"] == 2
    assert got["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_launch_count_per_training_step():
    # 1080p with 32-pixel tiles: 2040 tiles, 11 tile bits, 2 tile passes
    assert bench.launches_per_step(0, 11) == 18  # the L1 loss taken in the compositing forward
    assert bench.launches_per_step(0, 11, fused=False) == 23
    assert bench.launches_per_step(0, 17) == bench.launches_per_step(0, 11) + 1  # a third tile pass
    assert bench.launches_per_step(1, 11) == 1 + (1 + 6 + 6) + 2 + 2 + 1  # 64-bit keys: 6 passes


def test_algorithmic_bytes_grow_with_the_work():
    n, M, k = 3_000_000, 10_000_000, 16
    for stage in ("preprocess", "bin_sort", "preprocess_bwd", "preprocess_bwd_adam"):
        few = bench.algorithmic_bytes(stage, n, M, 6, k, n_vis=1_000_000)
        many = bench.algorithmic_bytes(stage, n, M, 6, k, n_vis=2_000_000)
        assert 0 < few < many, stage
    assert bench.algorithmic_bytes("bin_sort", n, 2 * M, 6, k, n_vis=10 ** 6) > \
        bench.algorithmic_bytes("bin_sort", n, M, 6, k, n_vis=10 ** 6)
    # dense Adam: every parameter and both moments read and written, whatever is visible
    assert bench.algorithmic_bytes("adam", n, M, 6, k) == n * ((3 + 3 + 4 + 1 + 3 * k) * 28 + 32)


def test_cpu_baseline_window_is_scaled_to_the_frame():
    # the reference arm's quarter-window step: per-pixel stages scaled by the frame's pixels over
    # the window's, so the estimate stays close to the full-view one
    from paper_2501_12369_gb300 import synth
    import oracle
    oracle.build()
    s = synth.cluster_scene(20_000, seed=3)
    cam = synth.fibonacci_cameras(8, 6.0, 1920, 1080, 1500.0)[2]
    full = bench.cpu_baseline(s, [cam], "half_cosine", 32, target_seconds=0.2)
    quarter = bench.cpu_baseline(s, [cam], "half_cosine", 32, target_seconds=0.2, window=(960, 0, 960, 544))
    assert full["value"] > 0 and quarter["value"] > 0
    assert "x4" in quarter["sample"] and "960x544 window at (960, 0)" in quarter["sample"]
    assert "one 1920x1080 view" in full["sample"]
    assert 0.2 < quarter["value"] / full["value"] < 5.0
