"""Host logic of the benchmark: the summary of the clock samples taken during the timed region
(median SM clock, maximum power, and the throttle reasons that make a run invalid), the
slowest-rank reduction on a single process, and the roofline entries (algorithmic flops per
launch over the launch's time, against the peak of the pipe the work runs on)."""
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


PEAKS = {"fp64_tflops": 1.25, "fp32_tflops": 80.0, "source": "test"}


def test_roofline_of_the_fused_kernel():
    """One launch holds both element kernels: its FP64 part is set against the FP64 peak and its
    FP32 part against the FP32 peak, both over the launch's own time; the DRAM traffic is the
    capture's for that kernel and workload."""
    E, ms = 937_860, 11.64
    out = bench.roofline_entries({"fused": ms, "fill": 0.05}, E, 1, False, PEAKS, "channel_re1000_mixed")
    assert [(r["kernel"], r["pipe"]) for r in out] == [("fused_assembly", "fp64"), ("fused_assembly", "fp32")]
    f64, f32 = out
    assert abs(f64["achieved"] - 24_300 * E / (ms * 1e-3) / 1e12) < 1e-12
    assert abs(f64["frac"] - f64["achieved"] / 1.25) < 1e-12
    assert abs(f32["achieved"] - 93_400 * E / (ms * 1e-3) / 1e12) < 1e-12
    assert abs(f32["frac"] - f32["achieved"] / 80.0) < 1e-12
    assert f64["traffic"] == bench.NCU_TRAFFIC_BYTES[("fused", "channel_re1000_mixed")]
    assert f64["executed_flops_per_element"] == bench.EXECUTED_FLOPS["fused_fp64"]
    assert f32["executed_flops_per_element"] is None


def test_roofline_of_the_two_kernel_forms():
    """FP64 mode: residual and tangent each on the FP64 pipe with their executed counts; mixed
    precision with two kernels: the tangent on the FP32 pipe; no traffic where no capture exists;
    the tetrahedron's single kernel on its executed count."""
    E = 32_768
    fp64 = bench.roofline_entries({"residual": 0.4, "tangent": 2.0}, E, 0, False, PEAKS, "cavity32_re400_fp64")
    assert [(r["kernel"], r["pipe"]) for r in fp64] == [("residual", "fp64"), ("tangent", "fp64")]
    assert fp64[0]["executed_flops_per_element"] == bench.EXECUTED_FLOPS["residual"]
    assert fp64[1]["executed_flops_per_element"] == bench.EXECUTED_FLOPS["tangent_fp64"]
    assert fp64[1]["traffic"] == bench.NCU_TRAFFIC_BYTES[("tangent", "cavity32_re400_fp64")]
    mixed = bench.roofline_entries({"residual": 0.4, "tangent": 0.3}, E, 1, False, PEAKS, "no_capture")
    assert [(r["kernel"], r["pipe"]) for r in mixed] == [("residual", "fp64"), ("tangent", "fp32")]
    assert all(r["traffic"] is None for r in mixed)
    tet = bench.roofline_entries({"tangent": 0.5}, 55_566, 1, True, PEAKS, "tetcavity21_re400_mixed")
    assert len(tet) == 1 and tet[0]["kernel"] == "tet_assembly"
    assert abs(tet[0]["achieved"] - bench.EXECUTED_FLOPS["tet"] * 55_566 / 0.5e-3 / 1e12) < 1e-12
