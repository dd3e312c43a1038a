"""Reduced-precision path (FP32 arithmetic, FP64 state/traces/RK accumulation) against the
FP64 oracle: every result reports its relative L2 error (printed, and appended as a JSON line
to the file the DG_PRECISION_LOG environment variable names, if set) and must stay within its
regression bound below.
"""
import json
import os

import numpy as np
import pytest

from helpers import gpu_solver, oracle_mesh, oracle_state, rel_l2, small_mixed, to_dev
from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# Regression bounds per case of the plain FP32 path (every contraction in FP32), about 3x the
# measured error. Its error is set by the conditioning of the residual: R_p = -c0^2 div u of a
# nearly divergence-free field is a small difference of three directional derivatives, each
# with FP32 rounding (measured on the 64^3 workload: the pressure row carries 2.6e-5 of the
# 2.65e-5, and the error scales with c0^2). With the divergence in FP64 (fp64_divergence = 1,
# box elements) the 1e-6 target is met and asserted below (TARGET).
BOUNDS = {
    "tgv_4x4x4_n3": 3e-5, "wake_16x16x16_n4": 1e-6, "tgv_8x8x8_n5_slab30": 6e-6,
    "padapt_6x6x6_curved": 1.5e-5, "tgv_5x5x5_n1_vreman_llf": 1e-6, "tgv_5x5x5_n2_vreman_llf": 5e-6,
    "tgv_5x5x5_n6_vreman_llf": 3e-4, "tgv_5x5x5_n7_vreman_llf": 3e-4,
    "tgv_4x4x4_n3_rk3_10_steps_update": 7e-6, "mixed_64x64x64_n4_sampled": 1e-4,
    "tgv_5x5x5_rotated_affine_mixed_orders": 1e-4, "padapt_5x5x5_one_sided_mixed_face": 5e-5,
    "padapt_5x5x5_kep": 5e-5, "wake_8x8x8_n4_kep": 1e-6,
    "channel_6x6x6_noslip": 1e-5, "channel_6x6x6_slip": 1e-5,
}


TARGET = 1e-6  # relative L2 residual error of the reduced-precision path (FP64 divergence)
DIV64 = {"fp64_divergence": 1}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _record(name, err):
    """Print the error; also append it as a JSON line to the file DG_PRECISION_LOG names, if set."""
    print(f"{name}: FP32 relative L2 error vs FP64 oracle = {err:.3e}")
    path = os.environ.get("DG_PRECISION_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": name, "rel_l2": err}) + "\n")


def _fp32_error(w, params=None, precision=1):
    M = oracle_mesh(w, params)
    q = oracle_state(w, M)
    R_ref = M.residual(q)
    S = gpu_solver(w, precision=precision, params=params)
    R = S.residual(to_dev(q)).cpu().numpy()
    return rel_l2(R, R_ref)


@pytest.mark.parametrize("name,make", [
    ("tgv_4x4x4_n3", lambda: wl.tgv_4x4x4_n3()),
    ("wake_16x16x16_n4", lambda: wl.wake_16x16x16_n4()),
    ("tgv_8x8x8_n5_slab30", lambda: wl.tgv_32x32x32_n5(n=8)),
    ("padapt_6x6x6_curved", lambda: wl.padapt_32x32x32(n=6)),
])
def test_fp32_residual_error(name, make):
    err = _fp32_error(make())
    _record(name, err)
    assert err <= BOUNDS[name], err


def test_fp32_every_order_and_vreman_llf():
    for N in (1, 2, 6, 7):
        w = small_mixed(wl.tgv_4x4x4_n3(n_elem_dir=5, order=N), seed=20 + N)
        err = _fp32_error(w, params=dict(w.params, nu=1e-2, closure=1, riemann=1))
        _record(f"tgv_5x5x5_n{N}_vreman_llf", err)
        assert err <= BOUNDS[f"tgv_5x5x5_n{N}_vreman_llf"], (N, err)


def test_fp32_rotated_affine_mixed_orders():
    # re-oriented elements: general affine metric (not diagonal), every face orientation,
    # mortars between orders 2..5
    import dataclasses
    w = wl.tgv_4x4x4_n3(n_elem_dir=5, order=3)
    mesh, _ = wl.rotate_elements(w.mesh, 11)
    w = small_mixed(dataclasses.replace(w, mesh=mesh), seed=12, orders=(2, 5))
    err = _fp32_error(w, params=dict(w.params, nu=1e-2))
    _record("tgv_5x5x5_rotated_affine_mixed_orders", err)
    assert err <= BOUNDS["tgv_5x5x5_rotated_affine_mixed_orders"]


def test_fp32_one_sided_mixed_face():
    w = small_mixed(wl.padapt_32x32x32(n=5), seed=14, orders=(2, 5))
    err = _fp32_error(w, params=dict(w.params, nu=1e-2, mixed_face=1))
    _record("padapt_5x5x5_one_sided_mixed_face", err)
    assert err <= BOUNDS["padapt_5x5x5_one_sided_mixed_face"]


def test_fp32_kep_split_form():
    w = small_mixed(wl.padapt_32x32x32(n=5), seed=15, orders=(2, 5))
    err = _fp32_error(w, params=dict(w.params, nu=1e-2, split=1))
    _record("padapt_5x5x5_kep", err)
    assert err <= BOUNDS["padapt_5x5x5_kep"]
    ww = wl.wake_16x16x16_n4(n=8)
    err = _fp32_error(ww, params=dict(ww.params, split=1))
    _record("wake_8x8x8_n4_kep", err)
    assert err <= BOUNDS["wake_8x8x8_n4_kep"]


@pytest.mark.parametrize("name,make", [
    ("tgv_8x8x8_n5_slab30", lambda: wl.tgv_32x32x32_n5(n=8)),
    ("wake_16x16x16_n4", lambda: wl.wake_16x16x16_n4()),
    ("padapt_6x6x6_curved", lambda: wl.padapt_32x32x32(n=6)),
])
def test_tf32x3_tensor_core_contraction(name, make):
    # precision 2: the inviscid D contractions on the tensor cores in 3xTF32. Its error against
    # the FP64 oracle is reported like the FP32 path's, and it differs from the FP32-FMA path
    # by no more than FP32 rounding does (both amplified by the residual's conditioning)
    w = make()
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    R_ref = M.residual(q)
    qd = to_dev(q)
    R_tc = gpu_solver(w, precision=2).residual(qd).cpu().numpy()
    R_32 = gpu_solver(w, precision=1).residual(qd).cpu().numpy()
    err = rel_l2(R_tc, R_ref)
    _record(name + "_tf32x3", err)
    assert err <= 1.5 * BOUNDS[name], err
    assert rel_l2(R_tc, R_32) <= 1e-6 + 2.0 * rel_l2(R_32, R_ref), rel_l2(R_tc, R_32)


def test_tf32x3_every_order_rk_steps():
    for N in (1, 2, 3, 6, 7):
        w = small_mixed(wl.tgv_4x4x4_n3(n_elem_dir=5, order=N), seed=30 + N)
        p = dict(w.params, nu=1e-2)
        err = _fp32_error(w, params=p, precision=2)
        _record(f"tgv_5x5x5_n{N}_tf32x3", err)
        assert err <= 3e-4, (N, err)
    w = wl.tgv_4x4x4_n3()
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    q0 = q.copy()
    g = np.zeros_like(q)
    qd, gd = to_dev(q), to_dev(g)
    gpu_solver(w, precision=2).rk_step(qd, gd, w.dt, w.steps)
    M.rk_step(q, g, w.dt, w.steps)
    err = rel_l2(qd.cpu().numpy() - q0, q - q0)
    _record("tgv_4x4x4_n3_rk3_10_steps_update_tf32x3", err)
    assert err <= 1.5 * BOUNDS["tgv_4x4x4_n3_rk3_10_steps_update"]


def test_plain_tf32_contrast():
    # precision 3: one TF32 product of operands rounded to 10 mantissa bits, reported against
    # the FP64 oracle beside FP32 and 3xTF32 on the precision-variant configuration (reduced)
    w = wl.tgv_32x32x32_n5(n=8)
    errs = {p: _fp32_error(w, precision=p) for p in (1, 2, 3)}
    _record("tgv_8x8x8_n5_slab30_tf32", errs[3])
    assert errs[3] > 10 * errs[2], errs  # the correction products matter
    assert errs[3] < 5e-2, errs


@pytest.mark.parametrize("wall", [3, 4])
def test_fp32_walls(wall):
    w = wl.channel_walls(n=6, wall=wall)
    name = "channel_6x6x6_" + ("noslip" if wall == 3 else "slip")
    err = _fp32_error(w, params=dict(w.params, nu=1e-2))
    _record(name, err)
    assert err <= BOUNDS[name], err


def test_fp32_rk3_ten_steps():
    w = wl.tgv_4x4x4_n3()
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    q0 = q.copy()
    g = np.zeros_like(q)
    qd, gd = to_dev(q), to_dev(g)
    S = gpu_solver(w, precision=1)
    S.rk_step(qd, gd, w.dt, w.steps)
    M.rk_step(q, g, w.dt, w.steps)
    err = rel_l2(qd.cpu().numpy() - q0, q - q0)  # error of the state change over 10 steps
    _record("tgv_4x4x4_n3_rk3_10_steps_update", err)
    assert err <= BOUNDS["tgv_4x4x4_n3_rk3_10_steps_update"]


def test_fp32_mixed_full_size_sampled():
    import torch
    from test_gpu_parity import _fourier_torch
    from oracle import oracle as orc
    w = wl.mixed_64x64x64_n4()
    M = oracle_mesh(w)
    xyz = torch.from_numpy(M.node_coords()).cuda()
    q = torch.zeros((4, M.total), dtype=torch.float64, device="cuda")
    q[1:] = _fourier_torch(w, xyz)
    q[1] += 1.0
    del xyz
    S = gpu_solver(w, precision=1)
    R = S.residual(q).cpu().numpy()
    qh = q.cpu().numpy()
    rng = np.random.default_rng(1)
    sel = np.concatenate([rng.choice(np.flatnonzero(w.flags), 24, replace=False),
                          rng.choice(np.flatnonzero(w.flags == 0), 24, replace=False)])
    m = w.mesh
    Mx = orc.Mesh(m.hex, m.geom, 1, w.orders, w.flags, orc.params(**w.params), m.bc_tag, extended=True)
    Rx = np.zeros_like(qh)
    Mx.residual(qh, sel=sel, out=Rx)
    idx = np.concatenate([np.arange(M.offsets[e], M.offsets[e + 1]) for e in sel])
    err = rel_l2(R[:, idx], Rx[:, idx])
    _record("mixed_64x64x64_n4_sampled", err)
    assert err <= BOUNDS["mixed_64x64x64_n4_sampled"]
    S.set_params(dict(w.params, **DIV64))
    R = S.residual(q).cpu().numpy()
    err = rel_l2(R[:, idx], Rx[:, idx])
    _record("mixed_64x64x64_n4_sampled_div64", err)
    assert err <= TARGET, err


@pytest.mark.parametrize("name,make", [
    ("tgv_4x4x4_n3", lambda: wl.tgv_4x4x4_n3()),
    ("wake_16x16x16_n4", lambda: wl.wake_16x16x16_n4()),
    ("tgv_8x8x8_n5_slab30", lambda: wl.tgv_32x32x32_n5(n=8)),
])
@pytest.mark.parametrize("precision", [1, 2])
def test_fp64_divergence_meets_the_target(name, make, precision):
    # box elements: the divergence in FP64, the rest of the momentum fluxes in FP32 FMAs
    # (precision 1) or 3xTF32 tensor-core contractions (precision 2)
    w = make()
    err = _fp32_error(w, params=dict(w.params, **DIV64), precision=precision)
    _record(f"{name}_div64" + ("_tf32x3" if precision == 2 else ""), err)
    assert err <= TARGET, err
    assert err < _fp32_error(w, precision=precision)  # and it is the more accurate mode


# Coarse Taylor-Green meshes at N >= 4 (elements of a quarter period or more): the velocity
# varies by O(|u|) across an element, so the deviation form gains nothing and the momentum rows'
# FP32 contractions carry ~20 eps_32 (the sum of |D_im f_m| over the result); measured 2.0e-6 at
# N = 4 (FP32) and 4.0e-6 (3xTF32) on 6^3. Bounds: about 3x the measured error.
COARSE_DIV64 = {("tgv_6x6x6_n4", 1): 6e-6, ("tgv_6x6x6_n4", 2): 1.2e-5}


@pytest.mark.parametrize("precision", [1, 2])
def test_fp64_divergence_coarse_high_order(precision):
    w = wl.tgv_4x4x4_n3(n_elem_dir=6, order=4)
    err = _fp32_error(w, params=dict(w.params, **DIV64), precision=precision)
    _record("tgv_6x6x6_n4_div64" + ("_tf32x3" if precision == 2 else ""), err)
    assert err <= COARSE_DIV64[("tgv_6x6x6_n4", precision)], err
    assert err < _fp32_error(w, precision=precision)


def test_fp64_divergence_every_order_mixed_flags():
    # the target holds for N <= 3 on this coarse 4^3 mesh; above, the bound of the coarse cases
    for N in (1, 2, 3, 4, 5, 6, 7):
        w = small_mixed(wl.tgv_4x4x4_n3(n_elem_dir=4, order=N), seed=40 + N)
        p = dict(w.params, nu=1e-2, **DIV64)
        err = _fp32_error(w, params=p)
        _record(f"tgv_4x4x4_n{N}_mixed_flags_div64", err)
        assert err <= (TARGET if N <= 3 else 2e-5), (N, err)


def test_fp64_divergence_rk_steps():
    w = wl.tgv_4x4x4_n3()
    p = dict(w.params, **DIV64)
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    q0 = q.copy()
    g = np.zeros_like(q)
    qd, gd = to_dev(q), to_dev(g)
    gpu_solver(w, precision=1, params=p).rk_step(qd, gd, w.dt, w.steps)
    M.rk_step(q, g, w.dt, w.steps)
    err = rel_l2(qd.cpu().numpy() - q0, q - q0)
    _record("tgv_4x4x4_n3_rk3_10_steps_update_div64", err)
    assert err <= TARGET, err
