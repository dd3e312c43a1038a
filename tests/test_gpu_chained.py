"""Chained Runge-Kutta steps (dg_rk_step with nsteps > 1): every stage's update writes the next
stage's face traces, so only the first step runs the trace kernel. The state after K chained
steps must be bitwise that of K calls with nsteps = 1, for every form and node set, and the
chained steps launch one kernel fewer per trace bucket."""
import numpy as np
import pytest

from helpers import gpu_solver, oracle_mesh, oracle_state, small_mixed, to_dev
from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    tgv = wl.tgv_4x4x4_n3(n_elem_dir=5, order=4)
    mixed = small_mixed(wl.padapt_32x32x32(n=5), seed=51, orders=(2, 5))
    return [
        ("fp64_lobatto", tgv, 0, {}),
        ("fp32_lobatto", tgv, 1, {}),
        ("fp32_mortars_curved", mixed, 1, {"nu": 1e-2}),
        ("tf32x3_fp64_divergence", tgv, 2, {"fp64_divergence": 1}),
        ("fp64_gauss_legendre", tgv, 0, {"nodes": 1}),
        ("fp64_wake_inflow_outflow", wl.wake_16x16x16_n4(n=6, order=3), 0, {}),
    ]


@pytest.mark.parametrize("name,w,precision,extra", _cases(), ids=[c[0] for c in _cases()])
def test_chained_steps_equal_single_steps(name, w, precision, extra):
    import torch
    p = dict(w.params, **extra)
    M = oracle_mesh(w, p)
    q = oracle_state(w, M)
    S = gpu_solver(w, precision=precision, params=p)
    dt = 1e-4
    qa, ga = to_dev(q), torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
    for _ in range(5):
        S.rk_step(qa, ga, dt, 1)
    single = S.launches_per_step
    qb, gb = to_dev(q), torch.zeros_like(ga)
    S.rk_step(qb, gb, dt, 5)
    S.check_device()
    assert torch.equal(qa, qb), float((qa - qb).abs().max())
    # the trace kernels (one per order bucket) are gone from the later steps
    assert 1 <= single - S.launches_per_chained_step < single, (single, S.launches_per_chained_step)
    # an odd and an even number of chained steps (both trace-buffer parities), then a single one
    qc, gc = to_dev(q), torch.zeros_like(ga)
    S.rk_step(qc, gc, dt, 2)
    S.rk_step(qc, gc, dt, 3)
    assert torch.equal(qa, qc)


def test_chained_compressible_form():
    import torch
    w = wl.cns_tgv(n=4, order=3)
    S = gpu_solver(w, precision=0)
    xyz = S.node_coords()
    u = torch.from_numpy(wl.cns_state(xyz.cpu().numpy(), w.seed, period=2 * np.pi)).cuda()
    ua, ga = u.clone(), torch.zeros_like(u)
    for _ in range(4):
        S.rk_step(ua, ga, w.dt, 1)
    ub, gb = u.clone(), torch.zeros_like(u)
    S.rk_step(ub, gb, w.dt, 4)
    S.check_device()
    assert torch.equal(ua, ub)
