"""Host-side logic of bench.py that decides whether a measurement stands: the clock record
(median SM clock, maximum, throttle reasons seen during the timed region), the reference arm's
contract line, and the roofline entries (their key, the lookup of the ncu record of the current
kernel sources, and their arithmetic, with the GPU calls faked). No GPU needed."""
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


# --- the roofline entries: key, record lookup and arithmetic, with the GPU calls faked ---------
class _FakeTensor:
    def __init__(self, shape):
        self.shape = shape

    def __setitem__(self, key, value):
        pass

    def to(self, dev):
        return self


class _FakeEvent:
    def __init__(self, enable_timing=True):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 1.0  # ms between the two events


class _FakeCuda:
    Event = _FakeEvent

    @staticmethod
    def synchronize():
        pass


class _FakeTorch:
    float32 = "float32"
    cuda = _FakeCuda

    @staticmethod
    def zeros(shape, dtype=None, device=None):
        return _FakeTensor(shape)

    @staticmethod
    def zeros_like(t):
        return _FakeTensor(t.shape)

    @staticmethod
    def from_numpy(a):
        return _FakeTensor(a.shape)


class _FakePlan:
    """chambolle_iterate runs ceil(iters / depth) launches of the tile-24 shape at depth 8."""

    def __init__(self):
        self.launches = 0

    def chambolle_iterate(self, gl, p1, p2, H, W, pitch, iters, stream=None):
        self.launches += -(-iters // 8)

    def stats(self):
        return {"last_temporal_block": 8, "last_tile": 24, "kernel_launches": self.launches}


class _FakeTv:
    @staticmethod
    def pitch_for(W):
        return W


def _roofline(monkeypatch, tmp_path, records, src_hash="cafe0123beef"):
    import json
    import types

    import numpy as np

    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(records))
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: src_hash)
    job = types.SimpleNamespace(f=np.zeros((512, 512), np.float32), dt=0.5, n_inner=300)
    return bench.measure_roofline(_FakeTv, _FakeTorch, _FakePlan(), "config1_512x512_K50_it300",
                                  job, "cuda:0", None, reps=5)


def test_roofline_uses_the_record_of_the_current_sources(monkeypatch, tmp_path):
    key = "config1_512x512_K50_it300/tile24/tb8/cafe0123beef"
    hbm, issue = _roofline(monkeypatch, tmp_path,
                           {key: {"dram_bytes": 40000, "warp_inst": 2_400_000, "iters": 8}})
    # 5 calls x 38 launches (300 = 37 x 8 + 4) in 1 ms: 5.263 us per launch of 300 x 5 / 190
    # iterations on average; 20 B per pixel-iteration
    n_launch = 5 * 38
    per_launch = 1e-3 / n_launch
    it = 300 * 5 / n_launch
    alg = 20 * 512 * 512 * it
    assert hbm["profile_key"] == key and hbm["traffic"] == 40000
    assert abs(hbm["per_launch_us"] - per_launch * 1e6) < 1e-9
    assert abs(hbm["algorithmic_bytes_per_launch"] - alg) < 1e-3
    assert abs(hbm["achieved"] - alg / per_launch / 1e9) < 1e-6
    assert hbm["peak"] == 6000.0 and abs(hbm["frac"] - hbm["achieved"] / 6000.0) < 1e-12
    # the captured launch ran 8 iterations; the average launch runs `it`
    inst = 2_400_000 * it / 8
    assert abs(issue["warp_inst_per_launch"] - inst) < 1e-6
    ipeak = 152 * 4 * 2000.0 * 1e6 / 1e9
    assert issue["peak"] == ipeak
    assert abs(issue["achieved"] - inst / per_launch / 1e9) < 1e-6
    assert abs(issue["thread_inst_per_px_iter"] - 32 * inst / (512 * 512 * it)) < 1e-9


def test_roofline_drops_counters_of_other_sources(monkeypatch, tmp_path):
    # a record keyed by another source hash (the kernel changed since the capture): no traffic,
    # no issue roofline, but the timed HBM figure stands
    old = "config1_512x512_K50_it300/tile24/tb8/0123456789ab"
    hbm, issue = _roofline(monkeypatch, tmp_path, {old: {"dram_bytes": 1, "warp_inst": 1, "iters": 8}})
    assert hbm["traffic"] is None and issue is None
    assert hbm["achieved"] > 0 and hbm["profile_key"].endswith("/cafe0123beef")


def test_committed_traffic_records_are_well_formed():
    # every committed record names a workload, a tile, a depth and a 12-digit source hash, and
    # holds positive counts
    import json
    import os
    import re

    recs = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")))
    assert recs
    for key, rec in recs.items():
        assert re.fullmatch(r"[A-Za-z0-9_]+/tile\d+/tb\d+/[0-9a-f]{12}", key), key
        assert rec["dram_bytes"] >= 0 and rec["warp_inst"] > 0 and rec["iters"] > 0, key
