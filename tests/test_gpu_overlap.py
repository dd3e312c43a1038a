"""Overlapped launches of the pipelined reduced-precision passes (dg_set_launch_overlap): the
viscous and inviscid launches carry programmatic stream serialisation, and the inviscid launch
after a viscous pass runs the Euler elements with no NS neighbour and no mortar face before it
waits for that pass. Every result must be bitwise that of plain launches: residuals, single and
chained RK steps, after a change of flags, with mortars, and for every contraction form."""
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
    mixed = wl.mixed_64x64x64_n4(n=12)
    return [
        # wall layer and wake NS, the rest Euler: most Euler elements are independent
        ("fp32_mixed", mixed, 1, {}),
        ("fp32_fp64_divergence", mixed, 1, {"fp64_divergence": 1}),
        ("tf32x3", mixed, 2, {}),
        ("fp32_all_euler", wl.mixed_64x64x64_n4(n=8, all_euler=True), 1, {}),
        ("fp32_all_ns", wl.mixed_64x64x64_n4(n=8, all_ns=True), 1, {}),
        # scattered flags: few independent elements, many tiles at the class boundaries
        ("fp32_random_flags", small_mixed(wl.tgv_4x4x4_n3(n_elem_dir=7, order=4), seed=7, flags_p=0.1), 1, {}),
        # p-adaptive curved mesh: mortar launches between the viscous and inviscid passes
        ("fp32_mortars_curved", small_mixed(wl.padapt_32x32x32(n=5), seed=51, orders=(2, 5)), 1, {"nu": 1e-2}),
    ]


def _run(S, q, dt, overlap):
    import torch
    S.set_launch_overlap(overlap)
    qd = to_dev(q)
    R = S.residual(qd).clone()
    g = torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
    S.rk_step(qd, g, dt, 1)
    S.rk_step(qd, g, dt, 4)  # chained: both trace-buffer parities
    S.check_device()
    return R, qd, g


@pytest.mark.parametrize("name,w,precision,extra", _cases(), ids=[c[0] for c in _cases()])
def test_overlapped_launches_give_identical_results(name, w, precision, extra):
    import torch
    p = dict(w.params, **extra)
    M = oracle_mesh(w, p)
    q = oracle_state(w, M)
    S = gpu_solver(w, precision=precision, params=p)
    dt = 1e-4
    Ra, qa, ga = _run(S, q, dt, True)
    Rb, qb, gb = _run(S, q, dt, False)
    Rc, qc, gc = _run(S, q, dt, True)  # and back: the step graphs were rebuilt both times
    for x, y, z in ((Ra, Rb, Rc), (qa, qb, qc), (ga, gb, gc)):
        assert torch.equal(x, y), float((x - y).abs().max())
        assert torch.equal(x, z)
    assert bool(torch.isfinite(qa).all())


def test_overlap_after_a_change_of_flags():
    # the independent entries are recomputed with the flags: new NS elements next to formerly
    # independent ones must make those wait
    import torch
    w = wl.mixed_64x64x64_n4(n=10)
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    S = gpu_solver(w, precision=1)
    rng = np.random.default_rng(3)
    flags = w.flags.copy()
    flags[rng.integers(0, w.n_elem, size=w.n_elem // 20)] = 1
    out = []
    for overlap in (True, False):
        S.set_flags(w.flags)
        S.set_launch_overlap(overlap)
        qd = to_dev(q)
        g = torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
        S.rk_step(qd, g, 1e-4, 2)
        S.set_flags(flags)
        S.rk_step(qd, g, 1e-4, 3)
        S.check_device()
        out.append(qd)
    assert torch.equal(out[0], out[1])


def test_overlap_argument_is_checked():
    import ctypes
    from paper_2403_05463_gb300 import dg
    S = gpu_solver(wl.tgv_4x4x4_n3(n_elem_dir=3, order=3), precision=1)
    st = dg.load().dg_set_launch_overlap(S.h, ctypes.c_int(2))
    assert dg.STATUS[st] == "DG_ERR_ARG"
