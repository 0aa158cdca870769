"""The benchmark's clock summary (CPU): samples inside the timed region's
wall-clock window are the ones reported, throttle reasons are collected from
them, and without timestamps inside the window every sample is used."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(t, sm, mx, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, "0", str(sm), str(mx), "700.5", "0x0000000000000000", *reasons])


def test_window_selects_timed_samples():
    sys.path.insert(0, ROOT)
    import bench
    t = 1_800_000_000.0
    lines = [_line(t + 0.00, 1500, 2032, ("Not Active", "Not Active", "Not Active", "Active")),  # warm-up
             _line(t + 0.05, 2032, 2032), _line(t + 0.10, 2032, 2032), _line(t + 0.15, 2010, 2032),
             _line(t + 0.30, 1200, 2032, ("Active", "Not Active", "Not Active", "Not Active"))]       # after
    s = bench.clock_summary(lines, t + 0.04, t + 0.2)
    assert s["samples"] == 3 and s["window"] == "timed"
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0 and s["reasons"] == []


def test_reasons_and_fallback_to_all_samples():
    sys.path.insert(0, ROOT)
    import bench
    t = 1_800_000_000.0
    lines = [_line(t, 1900, 2032, ("Not Active", "Not Active", "Not Active", "Active")),
             _line(t + 0.05, 1950, 2032), "garbage", ""]
    s = bench.clock_summary(lines, t + 10.0, t + 11.0)  # no sample inside the window
    assert s["samples"] == 2 and s["window"] == "warm-up and timed"
    assert s["sm_mhz"] == 1925.0 and s["reasons"] == ["sw_power_cap"]
    s = bench.clock_summary(lines, t - 1.0, t + 1.0)
    assert s["window"] == "timed" and s["reasons"] == ["sw_power_cap"]
    assert bench.clock_summary([], 0.0, 1.0)["sm_mhz"] is None


def test_sampler_names_the_gpu_by_uuid_and_flags_thin_windows():
    """nvidia-smi ignores CUDA_VISIBLE_DEVICES, so the sampler names its GPU by
    UUID; a summary over fewer than 10 samples says so."""
    sys.path.insert(0, ROOT)
    import bench
    sid = bench.gpu_smi_id(0)
    assert sid.startswith("GPU-") or sid == "0"  # "0" only without a CUDA device
    t = 1_800_000_000.0
    s = bench.clock_summary([_line(t + 0.01 * i, 2032, 2032) for i in range(3)], t - 1, t + 1)
    assert s["samples"] == 3 and "weak" in s
    s = bench.clock_summary([_line(t + 0.01 * i, 2032, 2032) for i in range(12)], t - 1, t + 1)
    assert s["samples"] == 12 and "weak" not in s
