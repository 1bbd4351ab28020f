"""Host-side logic of bench.py on CPU: the clock record parsed from nvidia-smi samples (median SM
clock, throttle reasons), the roofline arithmetic of the kernel classes, the launch count of a
batched solve against the ncu launch list it was read from, the measured-peak lookup and the
work counts the roofline rests on."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks(lines):
    c = bench.Clocks(0)
    c.proc = _Proc()
    c.lines = list(lines)
    return c.stop()


def test_clock_record_median_and_reasons():
    row = "0, {sm}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {cap}"
    out = _clocks([row.format(sm=2070, cap="Not Active"), row.format(sm=1980, cap="Active"),
                   row.format(sm=2070, cap="Not Active"), "garbage line", "0, [N/A], 2070, 1, 2, 3, 4, 5, 6"])
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    hot = _clocks(["0, 1500, 2070, 1300, 0x8, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    c = bench.Clocks(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_roofline_arithmetic():
    V, steps = 4096, 550
    r = bench.kernel_roofline("pass1_persistent", 10.0, steps, V, 6682.8)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(768 * V * steps / 10.0 / 1e6)
    r = bench.kernel_roofline("pass2_persistent", 10.0, steps, V, 6682.8)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(1.259, rel=1e-3)
    assert r["achieved"] == pytest.approx((1368 + 360) * V * steps / 10.0 / 1e9)
    assert bench.kernel_roofline("no such kernel", 1.0, 1, 1, 1.0) is None


def test_work_counts():
    # the counts quoted in the design notes and the bench line
    assert bench.REGEN_DF_OPS_SITE == 12224
    assert bench.FP32_OPS_PEAK_T == pytest.approx(40.27, rel=1e-3)
    assert bench.DW_BYTES == {"f64": 960, "f32_12": 384, "f32_18": 480}
    assert bench.DWGRAD_BYTES_SITE == 1104


def test_batch_launch_count_matches_the_launch_list():
    # the ncu launch list of one 12-source, k = 550, m = 20 batched solve counts 755 launches
    assert bench.batch_launches(12, 550, 20) == 755
    # without deflation the two projection pairs go, with the stepwise pass 1 it is 2k - 1 launches
    assert bench.batch_launches(12, 550, 0) == 755 - 12 * 4
    assert bench.batch_launches(12, 550, 20, persistent_pass1=False) == 755 - 1 + (2 * 550 - 1)
    # the launch list of one 48-sequence headline batch at k = 480 without deflation (stepwise pass 1:
    # its 128-site blocks exceed one resident grid) counts 2027 launches
    assert bench.headline_launches(480, m=0) == 2027


def test_measured_peaks_lookup(tmp_path, monkeypatch):
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            want = json.load(f)["hbm_gbs"]
        assert bench.peaks() == (want, "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
