"""Launch-shape autotuner of the reduced-precision passes (dg_autotune): every tile shape and
kernel choice it can make gives the same residual, choices round-trip through the cache file,
and a tuned solver still meets the FP32 error bounds against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_solver, oracle_mesh, oracle_state, rel_l2, small_mixed, to_dev
from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _device_name():
    import torch
    return torch.cuda.get_device_name(0)


def _forced_cache(path, choices):
    """choices: {(pass, N, geo): (tile_alt, bps, visc_alt)} for this device."""
    with open(path, "w") as f:
        for (ps, n, geo), (alt, bps, valt) in choices.items():
            f.write(f"{_device_name()}\t{ps}\t{n}\t{geo}\t{alt}\t{bps}\t{valt}\n")


def _box_mixed_orders():
    # axis-aligned boxes (geometry kind 0) with every order 1..7 and mixed flags
    w = wl.tgv_4x4x4_n3(n_elem_dir=6, order=3)
    return small_mixed(w, seed=41, orders=(1, 7))


def _rotated_affine():
    # re-oriented elements: general affine metric (geometry kind 1), orders 2..6
    w = wl.tgv_4x4x4_n3(n_elem_dir=5, order=3)
    mesh, _ = wl.rotate_elements(w.mesh, 17)
    return small_mixed(dataclasses.replace(w, mesh=mesh), seed=42, orders=(2, 6))


@pytest.mark.parametrize("make", [_box_mixed_orders, _rotated_affine])
def test_every_choice_gives_the_same_residual(make, tmp_path):
    w = make()
    p = dict(w.params, nu=1e-2)
    M = oracle_mesh(w, p)
    q = oracle_state(w, M)
    qd = to_dev(q)
    S = gpu_solver(w, precision=1, params=p)
    R_default = S.residual(qd).cpu().numpy()
    keys = sorted({(int(n), g) for n in np.unique(w.orders) for g in (0, 1)})
    for alt, bps, valt in [(1, 0, 0), (0, 1, 0), (1, 2, 1), (0, 2, 1)]:
        cache = tmp_path / f"tune_{alt}{bps}{valt}.txt"
        choices = {}
        for n, g in keys:
            choices[(0, n, g)] = (alt, bps, 0)
            choices[(1, n, g)] = (alt, bps, valt)  # the viscous pass's tile shape too
        _forced_cache(cache, choices)
        T = gpu_solver(w, precision=1, params=p)
        rep = T.autotune(str(cache))
        assert "cached" in rep and " ms" not in rep, rep
        R = T.residual(qd).cpu().numpy()
        # tile shape and grid leave every node's FP32 sums as they are; the two viscous
        # kernels may round differently in the last FP32 bits
        assert rel_l2(R, R_default) <= (1e-6 if valt else 1e-12), (alt, bps, valt, rel_l2(R, R_default))


def test_tuning_round_trip_and_accuracy(tmp_path):
    w = small_mixed(wl.padapt_32x32x32(n=5), seed=43, orders=(2, 5))
    p = dict(w.params, nu=1e-2)
    M = oracle_mesh(w, p)
    q = oracle_state(w, M)
    R_ref = M.residual(q)
    cache = tmp_path / "tune.txt"
    S = gpu_solver(w, precision=1, params=p)
    rep = S.autotune(str(cache))
    assert "inviscid" in rep and " ms" in rep, rep
    lines = cache.read_text().splitlines()
    assert lines and all(line.startswith(_device_name() + "\t") for line in lines)
    err = rel_l2(S.residual(to_dev(q)).cpu().numpy(), R_ref)
    assert err <= 5e-5, err  # the FP32 bound of this case family
    # a second solver takes the cached choices without timing
    T = gpu_solver(w, precision=1, params=p)
    rep2 = T.autotune(str(cache))
    assert "cached" in rep2 and " ms" not in rep2, rep2
    # RK steps after tuning: the captured step is rebuilt with the chosen launch shapes
    q0 = q.copy()
    g = np.zeros_like(q)
    qd, gd = to_dev(q), to_dev(g)
    T.rk_step(qd, gd, 1e-4, 3)
    M.rk_step(q, g, 1e-4, 3)
    err = rel_l2(qd.cpu().numpy() - q0, q - q0)  # the state change, at FP32 accuracy
    assert err <= 5e-5, err


def test_fp64_has_nothing_to_tune():
    S = gpu_solver(wl.tgv_4x4x4_n3(), precision=0)
    assert "no launch choices" in S.autotune()


def _stage_case(flags_p=0.3, n=10, order=4):
    # one (order, box) bucket, no mortars: the persistent stage kernel applies
    w = wl.tgv_4x4x4_n3(n_elem_dir=n, order=order)
    return small_mixed(w, seed=44, flags_p=flags_p)


STAGE_CHOICES = {0: "separate launches", 1: "one persistent kernel", 2: "one launch with tile queues"}


@pytest.mark.parametrize("flags_p", [0.0, 0.3, 1.0])
@pytest.mark.parametrize("order", [3, 4, 5])
def test_persistent_stage_kernel_matches_separate_launches(flags_p, order, tmp_path):
    # one launch per RK stage (the persistent kernel with a grid barrier, and the kernel with
    # tile queues) against the separate launches: the same device code per element, so the same
    # bits, whatever order the tiles run in
    import torch
    w = _stage_case(flags_p, order=order)
    p = dict(w.params, nu=1e-2)
    M = oracle_mesh(w, p)
    q = oracle_state(w, M)
    out = {}
    for fused in (0, 1, 2):
        cache = tmp_path / f"stage{fused}.txt"
        # default shapes for both passes (the stage kernels'), the stage choice forced
        _forced_cache(cache, {(0, order, 0): (0, 0, 0), (1, order, 0): (0, 0, 0), (2, order, 0): (fused, 0, 0)})
        S = gpu_solver(w, precision=1, params=p)
        rep = S.autotune(str(cache))
        assert STAGE_CHOICES[fused] in rep, rep
        qd, gd = to_dev(q), torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
        S.rk_step(qd, gd, 1e-4, 3)
        S.check_device()
        out[fused] = (qd.cpu().numpy(), S.launches_per_step)
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][0], out[2][0])
    # three stages: traces once, then one launch per stage instead of viscous + inviscid
    if flags_p > 0:
        assert out[1][1] == out[0][1] - 3, (out[0][1], out[1][1])
        assert out[2][1] == out[0][1] - 3, (out[0][1], out[2][1])
    # and against the oracle, at the FP32 accuracy of the state change
    q0 = q.copy()
    g = np.zeros_like(q)
    M.rk_step(q, g, 1e-4, 3)
    assert rel_l2(out[1][0] - q0, q - q0) <= 1e-4


@pytest.mark.parametrize("viscous_shape,extra", [(0, {}), (1, {}), (0, {"fp64_divergence": 1})])
def test_tile_queue_stage_kernel_chained_steps(viscous_shape, extra, tmp_path):
    # regional flags (wall layer and wake NS, most Euler elements independent of the viscous
    # pass), chained steps (the queues are reset by each launch's last block, across graph
    # replays), with overlapped and plain launches; the separate launches may use the other
    # viscous tile shape, the one-launch kernel always uses the default one; and the variant
    # with the FP64 divergence
    import torch
    w = wl.mixed_64x64x64_n4(n=12)
    p = dict(w.params, **extra)
    M = oracle_mesh(w, p)
    q = oracle_state(w, M)
    out = {}
    # (stage choice, split): separate launches; the queue kernel with every block starting on
    # the viscous queue, or 1x / 3x its share of the tiles (the rest start on inviscid tiles)
    for fused, vsplit in ((0, 0), (2, 0), (2, 1), (2, 3)):
        cache = tmp_path / f"q{fused}{vsplit}.txt"
        _forced_cache(cache, {(0, 4, 0): (0, 0, 0), (1, 4, 0): (viscous_shape, 0, 0), (2, 4, 0): (fused, vsplit, 0)})
        S = gpu_solver(w, precision=1, params=p)
        assert STAGE_CHOICES[fused] in S.autotune(str(cache))
        for overlap in (True, False):
            S.set_launch_overlap(overlap)
            qd, gd = to_dev(q), torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
            S.rk_step(qd, gd, 1e-4, 2)
            S.rk_step(qd, gd, 1e-4, 5)
            S.check_device()
            out[(fused, vsplit, overlap)] = qd
    ref = out[(0, 0, True)]
    for k, v in out.items():
        assert torch.equal(v, ref), k


def test_autotuner_times_the_persistent_stage_kernel(tmp_path):
    w = _stage_case(0.3)
    S = gpu_solver(w, precision=1, params=dict(w.params, nu=1e-2))
    cache = tmp_path / "t.txt"
    _forced_cache(cache, {(0, 4, 0): (0, 0, 0), (1, 4, 0): (0, 0, 0)})  # the stage choice is timed
    rep = S.autotune(str(cache))
    assert "stage N=4 geo=0" in rep and all(c.split()[-1] in rep for c in STAGE_CHOICES.values()), rep
    # not offered where it does not apply: mixed orders (several buckets, mortars)
    T = gpu_solver(_box_mixed_orders(), precision=1)
    assert "stage N=" not in T.autotune()
