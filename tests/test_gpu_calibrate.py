"""arbgpu_calibrate: the measured integer multiply-add and 8-bit warp-MMA rates are positive and lie
between loose physical bounds set by the device's SM count and maximum clock (a rate far outside
them means a micro-kernel's work was dropped or miscounted)."""
from __future__ import annotations

import pytest

pytestmark = pytest.mark.gpu


def test_calibrate_rates_are_physical():
    import paper_1901_04289_gb300 as arb
    cal = arb.default_context().calibrate()
    sms, mhz = cal["sm_count"], cal["max_clock_mhz"]
    assert sms > 0 and mhz > 0
    lanes_clk = sms * mhz * 1e6 / 1e12  # T (SM x clock) per second
    # 32-bit multiply-adds: between 8 and 256 per SM per clock
    assert 8 * lanes_clk < cal["imad_tops"] < 256 * lanes_clk, cal
    assert 4 * lanes_clk < cal["imad_wide_tops"] < 256 * lanes_clk, cal
    # 8-bit warp MMA: at least as many operations per SM per clock as the 32-bit multiply-adds
    # the same units could issue, and below 32768 (far above any dense 8-bit tensor rate)
    assert 8 * lanes_clk < cal["mma_s8_tops"] < 32768 * lanes_clk, cal
    assert arb.default_context().status() == 0
