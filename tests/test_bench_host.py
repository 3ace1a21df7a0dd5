"""bench.py's host-side pieces without a GPU: the clock sampler's parsing of
nvidia-smi lines (median clock, throttle reasons) and the stage work model's
arithmetic for the blend kernels."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_reports_median_and_active_reasons():
    cs = bench.ClockSampler(0)
    cs.proc = _Proc()
    cs.lines = [
        "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    out = cs.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_sampler_without_samples():
    cs = bench.ClockSampler(0)
    cs.proc = _Proc()
    assert cs.stop() is None


def test_blend_work_counts_blended_pairs():
    rz = types.SimpleNamespace(n=1000, layout=types.SimpleNamespace(tiles=300))
    work, blended = bench.stage_work(rz, (2500, 40000), 4, 10000, 123456)
    assert blended == 123456
    assert work["blend_forward"] == ("alu", bench.FWD_FLOP_PER_BLENDED * 123456, "FLOP")
    assert work["blend_backward"] == ("alu", bench.BWD_FLOP_PER_BLENDED * 123456, "FLOP")
    # 300 tiles: 9 bits, 2 passes, 2500 records (12-bit ids): packed, 28 B per entry and 20 B per record
    assert work["tile_sort"] == ("hbm", 28.0 * 40000 + 20.0 * 2500, "B")
    # 70,000 tiles (17 bits, 3 passes): unpacked, 8 B written by the duplication, 16 B per entry and pass
    rz3 = types.SimpleNamespace(n=1000, layout=types.SimpleNamespace(tiles=70000))
    work3, _ = bench.stage_work(rz3, (2500, 40000), 4, 10000, 1)
    assert work3["tile_sort"] == ("hbm", 8.0 * 40000 + 3 * 16.0 * 40000 - 4.0 * 40000 + 20.0 * 2500, "B")
