"""Host-side logic of bench.py (no GPU): the clock sampler's window and
summary, and the algorithmic Gram flop count behind the roofline."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

IDLE = "2032, 2032, 500.1, Not Active, Not Active, Not Active, Not Active"


def _sampler(lines, first, last):
    s = bench.ClockSampler()
    s.lines = list(lines)
    s.first, s.last = first, last
    return s


def test_clock_summary_uses_the_window_only():
    # The samples outside [first, last) (before the region's last preceding
    # sample, after its first following one) must not count.
    lines = ["345, 2032, 90.0, Not Active, Not Active, Not Active, Not Active",
             IDLE,
             "2017, 2032, 900.0, Not Active, Not Active, Not Active, Active",
             IDLE,
             "330, 2032, 80.0, Not Active, Active, Not Active, Not Active"]
    out = _sampler(lines, 1, 4).summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2032.0  # median of 2032, 2017, 2032
    assert out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == ["sw_power_cap"]  # the hw_thermal_slowdown sample lies outside


def test_clock_summary_flags_every_active_reason():
    line = "1500, 2032, 700.0, Active, Active, Active, Active"
    out = _sampler([line], 0, 1).summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    out = _sampler(["garbage", "1, 2"], 0, 2).summary()
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_gram_flops_is_the_sum_of_in2_jn_over_the_eig_modes():
    # Eq. 4: mode n of st-HOSVD forms an I_n x I_n Gram over J_n columns, J_n
    # the product of the current sizes of the other modes (modes before n
    # already truncated to their ranks).
    f = bench.gram_flops((640, 640, 640), (64, 64, 64), [0, 0, 0])
    assert f == 640.0**2 * (640 * 640) + 640.0**2 * (64 * 640) + 640.0**2 * (64 * 64)
    g = bench.gram_flops((128,) * 4, (16,) * 4, [0, 0, 0, 0])
    assert g == 128.0**2 * (128**3 + 16 * 128**2 + 16**2 * 128 + 16**3)
    # An ALS mode forms no Gram but still truncates its mode.
    h = bench.gram_flops((640, 640, 640), (64, 64, 64), [0, 1, 0])
    assert h == 640.0**2 * (640 * 640) + 640.0**2 * (64 * 64)
    # Another mode order changes which sizes are already truncated.
    k = bench.gram_flops((100, 200, 300), (10, 20, 30), [0, 0, 0], mode_order=[2, 0, 1])
    assert k == 300.0**2 * (100 * 200) + 100.0**2 * (200 * 30) + 200.0**2 * (10 * 30)
