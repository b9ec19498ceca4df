"""Host logic of the benchmark: the summary of the clock samples taken during the timed region
(median SM clock, maximum power, and the throttle reasons that make a run invalid), and the
slowest-rank reduction on a single process."""
import bench


def write_samples(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.p = object()  # as if the sampler had run and written its file
    s.path = str(tmp_path / "clocks.csv")
    (tmp_path / "clocks.csv").write_text("\n".join(lines) + "\n")
    return s


def test_clock_summary_median_power_and_reasons(tmp_path):
    s = write_samples(tmp_path, [
        "0, 2070, 2070, 210.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 250.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "a line that is not a sample",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["power_w_max"] == 380.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_every_throttle_reason(tmp_path):
    s = write_samples(tmp_path, [
        "0, 1500, 2070, 900.0, 0x0000000000000048, Active, Not Active, Not Active, Not Active",
        "0, 1400, 2070, 950.0, 0x0000000000000068, Active, Active, Active, Not Active",
    ])
    out = s.summary()
    assert out["sm_mhz"] == 1450.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_a_sampler_or_samples(tmp_path):
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]
    s = write_samples(tmp_path, ["no samples here"])
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}


def test_slowest_rank_on_one_process():
    assert bench.max_over_ranks(1.25) == 1.25
