"""Host-side helpers of bench.py that need no GPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fifo_latencies_closed_form():
    # the FP64 one-at-a-time estimate of the serving benchmark: arrivals at 0, 1, 2 s and
    # 1.5 s of service each queue up (1.5, 2.0, 2.5 s); an idle gap resets the queue
    lat = bench.fifo_latencies_ms([0.0, 1.0, 2.0, 10.0], [1.5, 1.5, 1.5, 0.5])
    assert lat.tolist() == pytest.approx([1500.0, 2000.0, 2500.0, 500.0])
    assert bench.fifo_latencies_ms([], []).size == 0


def test_lane_peak_is_the_derived_fp32_pipe_rate():
    # 152 SMs x 128 FP32 lanes x 2070 MHz, one lane operation per lane per cycle
    assert bench.LANE_PEAK_TOPS == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    assert 40.2 < bench.LANE_PEAK_TOPS < 40.3
