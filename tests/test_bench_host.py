"""Host-side logic of bench.py (no GPU): the algorithmic byte model behind `roofline` and the
clock-sample parsing behind `clocks`."""

import math
import os
import sys
import tempfile

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_byte_model_without_pruning_is_the_complex64_round_trips():
    # no sub-box (s = n = 2N): every pass reads and writes whole complex64 arrays
    N, n = 128, 256
    b = bench.algorithmic_bytes_per_rotation(n, N, 0)
    mb = {k: v / 1e6 for k, v in b.items()}
    assert math.isclose(mb["spread"], 8 * n ** 3 / 1e6)                  # grid written once
    assert round(mb["fwd_x"], 1) == 201.3 and round(mb["fwd_y"], 1) == 100.7
    assert round(mb["fused"], 1) == 67.1 and round(mb["inv_y"], 1) == 33.6 and round(mb["inv_x"], 1) == 16.8
    total = sum(b[k] for k in ("spread", "fwd_x", "fwd_y", "fused", "inv_y", "inv_x")) / 1e6
    assert abs(total - 553.648128) < 1e-9                          # 553.7 MB as a sum of rounded entries
    # the sample reads of the spread: 16-byte position + 8-byte weight per sample
    assert bench.algorithmic_bytes_per_rotation(n, N, 1000)["spread"] - b["spread"] == 24 * 1000
    # 2D: one forward column pass, no y passes
    b2 = bench.algorithmic_bytes_per_rotation(64, 32, 0, dim=2)
    assert "fwd_y" not in b2 and b2["fused"] == (64 * 32 + 2 * 32 * 32) * 8


def test_sub_box_bounds_the_rotated_moving_shape():
    # the spread never leaves the sub-box: radius in oversampled cells + half the kernel + margin
    for radius, N, L in ((1.82, 128, 10.9), (0.3, 64, 6.6), (40.0, 192, 153.6)):
        s = bench.sub_box(radius, N, L)
        n = 2 * N
        assert s % 2 == 0 and s <= n
        if s < n:
            assert s / 2 >= radius * n / L + 3
    assert bench.sub_box(1e3, 128, 10.9) == 256


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_parse_median_and_reasons():
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    cs.p = _Proc()
    rows = ["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
            "2055, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
            "1980, 2070, 1401.2, Not Active, Not Active, Not Active, Active",
            "garbage line",
            "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active"]
    cs.f.write("\n".join(rows) + "\n")
    out = cs.stop()
    assert out["sm_mhz"] == float(np.median([2070, 2055, 1980])) and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert not os.path.exists(cs.f.name)


def test_traffic_model_reproduces_its_captures_and_scales_per_rotation():
    # the DRAM bytes the bench reports as roofline.traffic: at the captured batch
    # the model returns the captured read + write bytes exactly; the product table's
    # bytes are charged once per launch and the rest per rotation; shapes without
    # a capture report None
    assert bench.traffic_per_launch("fused", 156, 192, 20) == 976803840 + 1081333248
    assert bench.traffic_per_launch("fused", 108, 128, 34) == 552969728 + 529623040
    once = 192 ** 3 * 8  # W' of the docking grid, complex64
    per = (976803840 + 1081333248 - once) / 20
    assert bench.traffic_per_launch("fused", 156, 192, 40) == round(40 * per + once)
    assert bench.traffic_per_launch("fused", 108, 128, 17) == round((552969728 + 529623040) / 2)
    assert bench.traffic_per_launch("fwd_y", 156, 192, 20) is None
    assert bench.traffic_per_launch("fused", 156, 192, None) is None


def test_every_fft_plan_has_a_description():
    # the bench names the plan it ran from the library's plan values (SD_FFT_*)
    assert sorted(bench.FFT_PLAN_TEXT) == [0, 1, 2, 3]
    assert all(isinstance(t, str) and t for t in bench.FFT_PLAN_TEXT.values())
