"""Host logic of bench.py: parsing the clock samples taken during the timed region and the rule
that rejects a timed region (and has it measured once more)."""
import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s.summary()


def test_clock_summary_parses_nvidia_smi_rows():
    rows = ["0, 2070, 2070, 810.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage line", ""]
    s = _sampler(rows)
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert _sampler([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_clock_rejection_rules():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 5}
    assert bench.clock_rejection(ok) is None
    assert bench.clock_rejection(dict(ok, reasons=["sw_power_cap"], sm_mhz=1500.0)) is None   # kept, noted
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert r in bench.clock_rejection(dict(ok, reasons=[r]))
    assert "no reason" in bench.clock_rejection(dict(ok, sm_mhz=1200.0))                      # a clock lock
    assert bench.clock_rejection(dict(ok, sm_mhz=1800.0)) is None
    assert bench.clock_rejection({"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}) is None
