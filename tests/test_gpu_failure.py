"""Failure detection of the pipelined reduced-precision passes, through the C ABI, without a GPU
fault: a test hook makes the producer warp of block 0 stop before a tile, so that block's
consumers wait for data that never comes. Their bounded wait must run out, record
DG_ERR_TIMEOUT with the site in the device error word, and return; the call completes and the
context stays usable (the next residual matches the oracle again)."""
import time

import numpy as np
import pytest

from helpers import gpu_solver, oracle_mesh, oracle_state, rel_l2, to_dev
from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SITES = {1: "inviscid consumers", 3: "viscous consumers"}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(flags_value, n=12):
    # 12^3 elements at N = 4: 864 inviscid tiles of two elements, more than the resident
    # blocks, so block 0 runs several tiles and stop_tile = 1 stops it after one full tile
    w = wl.tgv_4x4x4_n3(n_elem_dir=n, order=4)
    return w.with_flags(np.full(w.n_elem, flags_value, np.uint8))


@pytest.mark.parametrize("flags_value,site", [(0, 1), (1, 3)])
@pytest.mark.parametrize("stop_tile", [0, 1])
def test_bounded_wait_times_out_and_the_context_recovers(flags_value, site, stop_tile):
    import torch
    from paper_2403_05463_gb300 import dg
    w = _case(flags_value)
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    R_ref = M.residual(q)
    S = gpu_solver(w, precision=1)
    qd = to_dev(q)
    R_ok = S.residual(qd).cpu().numpy()
    err_ok = rel_l2(R_ok, R_ref)
    assert err_ok < 1e-3  # the plain FP32 path's error on this state (about 6e-5)
    # all-Euler: only the inviscid pass is pipelined here; all-NS: the viscous pass runs first
    S.set_wait_limit(polls=1 << 14, stop_tile=stop_tile)
    t0 = time.perf_counter()
    S.residual(qd)
    with pytest.raises(dg.DGError) as ei:
        S.check_device()
    elapsed = time.perf_counter() - t0
    assert dg.STATUS[ei.value.status] == "DG_ERR_TIMEOUT", str(ei.value)
    assert f"site {site}" in str(ei.value), (str(ei.value), SITES[site])
    assert elapsed < 30.0
    # the error word was cleared, the context is usable, the default budget is back
    S.set_wait_limit(0, -1)
    S.check_device()
    R = S.residual(qd).cpu().numpy()
    S.check_device()
    assert rel_l2(R, R_ref) == pytest.approx(err_ok, rel=1e-6, abs=1e-12)
    torch.cuda.synchronize()


def test_wait_limit_arguments_are_checked():
    from paper_2403_05463_gb300 import dg
    S = gpu_solver(_case(1, n=4), precision=1)
    for polls, stop in ((-1, -1), (1 << 31, -1), (0, -3)):
        with pytest.raises(dg.DGError) as ei:
            S.set_wait_limit(polls, stop)
        assert dg.STATUS[ei.value.status] == "DG_ERR_ARG"


def test_step_graph_is_rebuilt_after_the_limit_changes():
    # the captured RK step holds the launch arguments: a step after the hook is switched on
    # must time out, and one after it is switched off must match an uninterrupted run
    import torch
    from paper_2403_05463_gb300 import dg
    w = _case(0)
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    S = gpu_solver(w, precision=1)
    qa, ga = to_dev(q), torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
    S.rk_step(qa, ga, w.dt, 1)  # capture the step graph
    S.check_device()
    S.set_wait_limit(polls=1 << 14, stop_tile=0)
    qb, gb = to_dev(q), torch.zeros_like(ga)
    S.rk_step(qb, gb, w.dt, 1)
    with pytest.raises(dg.DGError) as ei:
        S.check_device()
    assert dg.STATUS[ei.value.status] == "DG_ERR_TIMEOUT"
    S.set_wait_limit(0, -1)
    qc, gc = to_dev(q), torch.zeros_like(ga)
    S.rk_step(qc, gc, w.dt, 1)
    S.check_device()
    assert torch.equal(qc, qa)


def test_grid_barrier_of_the_persistent_stage_kernel_times_out(tmp_path):
    # block 0 of the one-kernel stage skips its grid-barrier arrival: every block's bounded wait
    # runs out (site 5), the step returns, the barrier is reset, and the next step is exact
    import torch
    from paper_2403_05463_gb300 import dg
    w = _case(1, n=10)
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    S = gpu_solver(w, precision=1)
    cache = tmp_path / "stage.txt"
    with open(cache, "w") as f:
        for ps, choice in ((0, "0\t0\t0"), (1, "0\t0\t0"), (2, "1\t0\t0")):
            f.write(f"{torch.cuda.get_device_name(0)}\t{ps}\t4\t0\t{choice}\n")
    assert "one persistent kernel" in S.autotune(str(cache))
    qa, ga = to_dev(q), torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
    S.rk_step(qa, ga, w.dt, 1)
    S.check_device()
    S.set_wait_limit(polls=1 << 12, stop_tile=-2)
    qb, gb = to_dev(q), torch.zeros_like(ga)
    t0 = time.perf_counter()
    S.rk_step(qb, gb, w.dt, 1)
    with pytest.raises(dg.DGError) as ei:
        S.check_device()
    assert time.perf_counter() - t0 < 30.0
    assert dg.STATUS[ei.value.status] == "DG_ERR_TIMEOUT" and "site 5" in str(ei.value), str(ei.value)
    S.set_wait_limit(0, -1)
    qc, gc = to_dev(q), torch.zeros_like(ga)
    S.rk_step(qc, gc, w.dt, 1)
    S.check_device()
    assert torch.equal(qc, qa)


def test_tile_queue_stage_kernel_wait_times_out(tmp_path):
    # the one-launch stage kernel with tile queues: block 0's producer stops before its first
    # viscous tile, so the tiles it claimed never finish. The inviscid tiles that read viscous
    # results wait on the counter of finished viscous tiles; that bounded wait runs out (site 6)
    # unless block 0's consumers' wait (site 3) ran out first. The step returns, the queues are
    # reset, and the next step is exact.
    import torch
    from paper_2403_05463_gb300 import dg
    w = _case(1, n=10)
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    S = gpu_solver(w, precision=1)
    cache = tmp_path / "queue.txt"
    with open(cache, "w") as f:
        for ps, choice in ((0, "0\t0\t0"), (1, "0\t0\t0"), (2, "2\t0\t0")):
            f.write(f"{torch.cuda.get_device_name(0)}\t{ps}\t4\t0\t{choice}\n")
    assert "one launch with tile queues" in S.autotune(str(cache))
    qa, ga = to_dev(q), torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
    S.rk_step(qa, ga, w.dt, 2)
    S.check_device()
    S.set_wait_limit(polls=1 << 12, stop_tile=0)
    qb, gb = to_dev(q), torch.zeros_like(ga)
    t0 = time.perf_counter()
    S.rk_step(qb, gb, w.dt, 1)
    with pytest.raises(dg.DGError) as ei:
        S.check_device()
    assert time.perf_counter() - t0 < 30.0
    assert dg.STATUS[ei.value.status] == "DG_ERR_TIMEOUT", str(ei.value)
    assert any(f"site {k}" in str(ei.value) for k in (1, 3, 6)), str(ei.value)
    S.set_wait_limit(0, -1)
    qc, gc = to_dev(q), torch.zeros_like(ga)
    S.rk_step(qc, gc, w.dt, 2)
    S.check_device()
    assert torch.equal(qc, qa)
