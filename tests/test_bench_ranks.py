"""CPU tests of bench.py's multi-rank path (one replica per rank, no collective on the data
path): two gloo ranks on 127.0.0.1 take the maximum of their step times, as the benchmark line
reports it, and under torchrun the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        slowest = bench.allmax(world, ms[rank])
        bench.barrier(world)
    finally:
        dist.destroy_process_group()
    q.put((rank, slowest))


def test_two_gloo_ranks_report_the_slowest_step():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ms = [4.75, 4.69]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert got == [(0, 4.75), (1, 4.75)]
    assert all(p.exitcode == 0 for p in procs)


def test_single_rank_allmax_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.allmax(1, 3.25) == 3.25


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    # a rank other than 0 exits 0 without work and prints nothing
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.main()
    assert rc == 0 and buf.getvalue() == ""


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
