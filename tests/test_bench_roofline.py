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


def test_traffic_records_follow_the_kernel_sources_and_the_launch():
    sys.path.insert(0, ROOT)
    import bench
    args = ("mixed_64x64x64_n4", "fp32", None, "inviscid_update", "tile_queues")
    for record in (bench.TRAFFIC_RECORD, bench.TRAFFIC_RECORD_CHAINED):
        text = open(record).read()
        if bench.kernel_sources_sha256() in text:
            assert bench.recorded_traffic(*args, record) > 0
        else:  # counters taken on other sources are not reported
            assert bench.recorded_traffic(*args, record) is None
    # other workloads, precisions, sizes, kernels or launch forms have no record
    assert bench.recorded_traffic("tgv_32x32x32_n5", *args[1:]) is None
    assert bench.recorded_traffic(args[0], "fp64", *args[2:]) is None
    assert bench.recorded_traffic(args[0], args[1], 32, *args[3:]) is None
    assert bench.recorded_traffic(*args[:4], "separate") is None


def test_stage_choice_reads_the_autotuner_report():
    sys.path.insert(0, ROOT)
    import bench
    head = "inviscid N=4 geo=0: 2 elements/tile, 0 blocks/SM (0 = max)\n"
    q = ("stage N=4 geo=0: one launch with tile queues: 1.5603 ms (one persistent kernel 1.6516 ms, "
         "one launch with tile queues 1.5603 ms, separate 1.6329 ms)")
    p = ("stage N=4 geo=0: one persistent kernel: 1.60 ms (one persistent kernel 1.60 ms, "
         "one launch with tile queues 1.70 ms, separate 1.65 ms)")
    s = ("stage N=4 geo=0: separate launches: 1.60 ms (one persistent kernel 1.70 ms, "
         "one launch with tile queues 1.75 ms, separate 1.60 ms)")
    assert bench.stage_choice(head + q) == "tile_queues"
    assert bench.stage_choice(head + p) == "persistent"
    assert bench.stage_choice(head + s) == "separate"
    assert bench.stage_choice(head) == "separate"
    # choices read from a tuning cache
    assert bench.stage_choice(head + "stage N=4 geo=0: cached, one launch with tile queues (split 3)") == "tile_queues"
    assert bench.stage_choice(head + "stage N=4 geo=0: cached, one persistent kernel (split 0)") == "persistent"
    assert bench.stage_choice(head + "stage N=4 geo=0: cached, separate launches (split 0)") == "separate"
