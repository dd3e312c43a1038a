"""CPU test of bench.py's roofline over the timed region: the one-launch stage kernel in a
chained call (every stage writes the next stage's traces, one trace-kernel launch first)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_timed_region_roofline_counts_every_launch_and_the_chained_trace_writes():
    sys.path.insert(0, ROOT)
    import bench
    # per-stage model: 6.0 GB in the stage kernel (two of three stages writing traces) and a
    # trace phase of 0.9 GB per stage (a third of a 1.35 GB read and a 1.35 GB write)
    ph_ms = {"traces": 0.2, "inviscid_update": 1.5}
    ph_bytes = {"traces": 0.9e9, "inviscid_update": 6.0e9}
    steps, ms_step, hbm = 10, 4.7, 6800.0
    r = bench.timed_region_roofline(ph_ms, ph_bytes, ms_step, steps, hbm)
    assert r["launches"] == 30
    # the region less one trace-kernel launch, over the stage launches
    assert r["ms_per_launch"] == pytest.approx((4.7 * 10 - 0.2) / 30)
    # each launch also writes a third of the 1.35 GB of traces that stage 2 adds
    assert r["bytes_per_launch"] == pytest.approx(6.0e9 + 1.35e9 / 3)
    assert r["achieved"] == pytest.approx(r["bytes_per_launch"] / (r["ms_per_launch"] * 1e-3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / hbm)
