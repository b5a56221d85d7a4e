"""Host-side logic of the benchmark (CPU): the clock and throttle-reason
summary of the nvidia-smi samples, and the rule that the roofline's DRAM
traffic comes from the committed ncu summary only while the near-field
kernel's sources are the ones it was captured on."""
import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_clock_summary_median_max_and_reasons():
    s = _sampler([
        "2070, 2070, 410.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 880.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 900.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "[N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_flags_thermal_and_hw_slowdown():
    s = _sampler([
        "1800, 2070, 1300, 0x48, Active, Not Active, Active, Not Active",
        "1700, 2070, 1300, 0x48, Not Active, Active, Not Active, Not Active",
    ])
    out = s.summary()
    assert out["sm_mhz"] == 1750.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    assert _sampler([]).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_near_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    digest = bench.near_source_digest()
    good = tmp_path / "good.md"
    good.write_text(f"traffic_bytes_per_launch: 12345\nsource_digest: {digest}\n")
    monkeypatch.setattr(bench, "NEAR_PROFILE", str(good))
    assert bench.near_traffic()[0] == 12345
    stale = tmp_path / "stale.md"
    stale.write_text("traffic_bytes_per_launch: 12345\nsource_digest: 0123456789abcdef\n")
    monkeypatch.setattr(bench, "NEAR_PROFILE", str(stale))
    t, note = bench.near_traffic()
    assert t is None and "changed" in note
    bare = tmp_path / "bare.md"
    bare.write_text("no figures here\n")
    monkeypatch.setattr(bench, "NEAR_PROFILE", str(bare))
    assert bench.near_traffic()[0] is None
    monkeypatch.setattr(bench, "NEAR_PROFILE", str(tmp_path / "missing.md"))
    assert bench.near_traffic() == (None, "no ncu summary")

