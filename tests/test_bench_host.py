"""Host-side logic of bench.py that decides whether a measurement stands: the clock record
(median SM clock, maximum, throttle reasons seen during the timed region). No GPU needed."""
import bench

FIELDS = "{i}, {sm}, {mx}, 500.0, 0x0, {hw}, {hwt}, {swt}, {pc}"


def _line(sm, mx=2070, hw="Not Active", hwt="Not Active", swt="Not Active", pc="Not Active"):
    return FIELDS.format(i=0, sm=sm, mx=mx, hw=hw, hwt=hwt, swt=swt, pc=pc)


def _summary(lines):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    return c.summary()


def test_median_clock_and_no_reasons():
    s = _summary([_line(2070), _line(2070), _line(1995)])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_every_throttle_reason_is_reported():
    s = _summary([_line(2070), _line(1800, hw="Active"), _line(1700, hwt="Active"),
                  _line(1900, swt="Active"), _line(2000, pc="Active")])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                            "sw_thermal_slowdown"]
    assert s["samples"] == 5 and s["sm_mhz"] == 1900.0


def test_malformed_and_missing_samples():
    s = _summary(["", "garbage", "0, [N/A], 2070, 1, 0x0, a, b, c, d", _line(2050)])
    assert s["samples"] == 1 and s["sm_mhz"] == 2050.0
    assert _summary([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_reference_arm_prints_the_contract_line():
    # `bench.py --impl reference` runs the FP64 oracle on the host: one JSON line with the
    # fields of the bench contract (a tiny sample here: two ROF steps of the 512^2 image)
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3", "--ref-steps-k", "2"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["config"]["workload"] == "config1_512x512_K50_it300"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
