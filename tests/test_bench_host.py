"""CPU checks of bench.py's host logic: the nvidia-smi clock record that
decides whether a timed run is kept (median SM clock, throttle reasons), the
algorithmic flop count behind the roofline fraction, the whole-job
throughput, and the peak denominators."""
import os

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _record(lines, tmp_path):
    c = bench.Clocks(0)
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    c.path, c.f, c.proc = str(p), open(os.devnull, "w"), _Proc()
    return c.stop()


OK = "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
CAP = "0, 1965, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
HOT = "0, 1500, 2070, 1400.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"


def test_clock_record_median_and_reasons(tmp_path):
    r = _record([OK, OK, CAP], tmp_path)
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    # a thermal slowdown is reported; unparsable lines are skipped
    r = _record([OK, HOT, "not a sample", "0, [N/A], 2070, 1.0, 0x0, a, b, c, d"], tmp_path)
    assert r["reasons"] == ["hw_thermal_slowdown"] and r["samples"] == 2 and r["sm_mhz"] == 1785.0


def test_clock_record_without_nvidia_smi():
    assert bench.Clocks(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_structured_flops_per_unit_and_epilogues():
    """One butterfly unit (N = 2), one level, one column: 8 r^2 + 36 r flops
    for the H form and 8 r^2 + 44 r for the G form (972 and 1044 at r = 9);
    the V^0 prologue adds 6 r, the switch 8 r^2 and U^L 8 r per point and
    column."""
    assert bench.structured_flops(1, 9, 2, 1, None, None, False) == 972
    assert bench.structured_flops(1, 9, 2, 1, None, None, True) == 1044
    N, nc, r = 1 << 10, 3, 9
    base = bench.structured_flops(4, r, N, nc, None, None, False)
    assert base == 4 * (N // 2) * nc * 972
    assert bench.structured_flops(4, r, N, nc, "V", None, False) - base == 6 * r * N * nc
    assert bench.structured_flops(4, r, N, nc, None, "switch", False) - base == 8 * r * r * N * nc
    g = bench.structured_flops(3, r, N, nc, None, None, True)
    assert bench.structured_flops(3, r, N, nc, None, "U", True) - g == 8 * r * N * nc


def test_throughput_and_peaks():
    # weak scaling: every rank's vectors count, divided by the slowest rank's time
    assert bench.job_throughput(64, 10, 2, 1000.0) == 1280.0
    assert bench.max_over_ranks(12.5, 1) == 12.5
    d, src = bench.peaks()
    assert src in ("measured", "fallback")
    assert d["hbm_gbs"] > 1000.0


def test_reference_arm_line(tmp_path):
    """`bench.py --impl reference` times the oracle on the host cores and
    prints one JSON line with the base contract's keys (small N here); a
    rank other than 0 prints nothing and exits 0."""
    import json
    import subprocess
    import sys
    cmd = [sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
           "--warmup", "3", "--N", "4096"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=str(tmp_path))
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    env = dict(os.environ, RANK="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=str(tmp_path), env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_fused_schedule_and_dominant_roofline():
    """The bench's copy of the launch schedule (levels 1..h and h+1..L in
    balanced chunks of at most k levels) and the dominant launch it picks
    from a per-launch profile."""
    import bench
    assert bench.fused_schedule(20, 10, 4) == [(0, 4, "H"), (4, 7, "H"), (7, 10, "H"), (10, 14, "G"), (14, 17, "G"),
                                               (17, 20, "G")]
    assert bench.fused_schedule(11, 5, 4) == [(0, 3, "H"), (3, 5, "H"), (5, 8, "G"), (8, 11, "G")]
    # two applies; the switch launch (7..10) is the longest in total
    prof = [(4, 3.0), (4, 2.0), (4, 3.5), (5, 3.1), (5, 2.1), (5, 2.2)] * 2
    d = bench.dominant_roofline(prof, 20, 10, 4, 9, 1 << 20, 64, 80.0, 6800.0)
    assert (d["lo"], d["hi"], d["kind"], d["epi"], d["n"]) == (7, 10, "H", "switch", 2)
    assert abs(d["avg_ms"] - 3.5) < 1e-12
    assert d["flops"] == bench.structured_flops(3, 9, 1 << 20, 64, None, "switch", False)
    assert abs(d["alu_frac"] - d["flops"] / 3.5e-3 / 1e12 / 80.0) < 1e-12


def test_apply_flops_is_the_sum_over_launches():
    """The whole-apply flop count used for the batch roofline equals the sum of
    the per-launch counts over any fusion depth's schedule."""
    import bench
    for L, k, nc in ((20, 4, 64), (11, 5, 3), (16, 3, 17)):
        h, N = L // 2, 1 << L
        tot = 0
        for lo, hi, kd in bench.fused_schedule(L, h, k):
            pro = "V" if lo == 0 else None
            epi = "U" if hi == L else ("switch" if hi == h else None)
            tot += bench.structured_flops(hi - lo, 9, N, nc, pro, epi, kd == "G")
        assert tot == bench.apply_flops(L, 9, N, nc)
