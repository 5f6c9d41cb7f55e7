"""Host logic of bench.py: parsing the clock samples taken during the timed region and the rule
that rejects a timed region (and has it measured once more)."""
import os

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


def test_headline_is_one_short_line_with_the_contract_keys():
    """The benchmark ends with one compact JSON line: the contract keys, a roofline of the dominant
    kernel, the CPU baseline and the end-to-end figure, a few KB at most (side measurements go to
    earlier lines)."""
    import json
    roof = {"kernel": "trace_2_replay", "bound": "alu", "achieved": 0.6312345678, "peak": 80.5, "unit": "TFLOP/s",
            "frac": 0.00784123, "traffic": None, "peak_basis": "nominal FP32", "ms_per_launch": 0.047,
            "share": 0.31, "rays_per_s": 1e10, "flops_per_launch": 3e7}
    cpu = {"value": 5900.123, "unit": "paths/s", "cores": 1, "kind": "oracle", "sample": "x" * 200,
           "multicore": {"value": 94000.0, "cores": 16}}
    e2e = {"value": 6.9e8, "unit": "paths/s", "h2d_bytes_per_step": 786432, "d2h_bytes_per_step": 8,
           "iters_per_s": 880.0, "last_loss": 0.01}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 9, "remeasured": None}
    variants = {"hit_store": {"ms_per_step": 0.72, "paths_evaluated_per_s": 1.09e9, "traced_paths_per_s": 7.3e8},
                "batched_64": {"ms_graph": 35.3, "ms_loop_plain": 64.1, "speedup": 1.81},
                "dsphere1024": {"ms_per_iter": 22.8, "paths_per_s": 1.66e9}, "volume256_meta": {"ms_per_iter": 9.09}}
    hbm = {"update_67M": {"frac": 0.98, "achieved": 6500.0, "unit": "GB/s"},
           "scatter_1024": {"frac": 0.32, "achieved": 2150.0, "unit": "GB/s"}}
    line = bench.headline(7.123456789e8, 20, 5, 1, 1.1034567, 906.2, roof, cpu, e2e, clocks, 1500, variants, hbm,
                          "measured")
    text = json.dumps(line, separators=(",", ":"))
    assert len(text) < 4096 and "\n" not in text
    back = json.loads(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in back, k
    assert back["value"] == 7.123e8 and back["config"]["workload"] == "spiral256"
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in back["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in back["e2e"], k
    assert back["steps"] * back["ms_per_step"] < 60e3


def test_fp32_peak_and_recorded_traffic_rules():
    """The ALU peak is computed from the device's SM count and clock; a recorded DRAM traffic
    figure is reported only while the traversal source is the one it was captured from."""
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54) < 0.01
    assert abs(bench.fp32_peak_tflops(148, 1965.0) - 148 * 256 * 1965e6 / 1e12) < 1e-9
    import hashlib
    with open(os.path.join(bench.ROOT, "paper_2309_15676_gb300", "csrc", "trace.cu"), "rb") as f:
        same = hashlib.sha1(f.read()).hexdigest() == bench.TRACE_DRAM["trace_cu_sha1"]
    assert bench.trace_traffic("trace_2_primal") == (bench.TRACE_DRAM["bytes"]["trace_2_primal"] if same else None)
    saved = dict(bench.TRACE_DRAM)
    try:
        bench.TRACE_DRAM.update({"source": "x", "trace_cu_sha1": "0" * 40, "bytes": {"trace_1_primal": 1.0}})
        assert bench.trace_traffic("trace_1_primal") is None      # source changed since the capture
        assert bench.trace_traffic("other") is None
    finally:
        bench.TRACE_DRAM.clear()
        bench.TRACE_DRAM.update(saved)


def test_reference_config_equals_the_gpu_arms():
    """Both arms name the same workload, with the paths per iteration of 12 traversals per pixel."""
    c = bench.workload_config(1)
    assert c["workload"] == "spiral256" and c["paths_per_iter"] == 12 * 256 * 256
    assert c["max_depth"] == 5 and (c["spp_prop"], c["spp_fd"]) == (2, 1)
