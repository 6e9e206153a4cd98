"""Host logic of bench.py: the clock-sample summary (no GPU, no nvidia-smi)."""
import bench

LINE = "0, {sm}, 2070, {pw}, 0x0, Not Active, Not Active, {swt}, {cap}"


def _lines(spec):
    return [(t, LINE.format(sm=sm, pw=pw, swt=swt, cap=cap)) for t, sm, pw, swt, cap in spec]


def test_clock_summary_keeps_the_timed_window():
    lines = _lines([(0.9, 345, 90, "Not Active", "Not Active"),      # before the region
                    (1.01, 2070, 600, "Not Active", "Active"),
                    (1.03, 2055, 650, "Not Active", "Not Active"),
                    (1.05, 2070, 640, "Not Active", "Not Active"),
                    (1.20, 1000, 100, "Active", "Not Active")])       # after it
    c = bench.clock_summary(lines, 1.0, 1.1, 20)
    assert c["samples"] == 3 and c["window"] == "timed region"
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["power_w_max"] == 650.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_summary_falls_back_to_the_next_sample():
    lines = _lines([(0.5, 2070, 90, "Not Active", "Not Active"),
                    (1.2, 1980, 500, "Active", "Not Active"),
                    (1.4, 2070, 500, "Not Active", "Not Active")])
    c = bench.clock_summary(lines, 1.0, 1.1, 20)
    assert c["samples"] == 1 and c["window"] == "first sample after the timed region"
    assert c["sm_mhz"] == 1980.0 and c["reasons"] == ["sw_thermal_slowdown"]


def test_clock_summary_skips_malformed_lines():
    lines = [(1.05, "0, [N/A], 2070, 100, 0x0, Not Active, Not Active, Not Active, Not Active"),
             (1.06, "garbage")]
    c = bench.clock_summary(lines, 1.0, 1.1, 20)
    assert c["samples"] == 0 and c["sm_mhz"] is None
