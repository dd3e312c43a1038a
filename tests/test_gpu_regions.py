"""Region detection on the GPU (dg_detect_regions, Sec. 2.1) against the FP64 oracle, through
the C ABI: node features, node memberships, element means and flags.

Tolerances: features are products of two (Q_S, Q_Omega) or three (R_S) gradient entries, so
their rounding is relative to max|J|^2 and max|J|^3 over the mesh; the bar is 1e-12 of those.
Memberships and their element means are probabilities, compared at 1e-11 absolute (the
log-weights a_k carry ~1e-16 |a_k| of rounding and dp/da <= 1/4). Flags must agree wherever the
two means differ by more than 1e-9; closer calls may go either way and are only checked to be
0 or 1."""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_solver, oracle_mesh, oracle_state, small_mixed, to_dev
from oracle import regions as rg
from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FEAT_TOL = 1e-12
PROB_TOL = 1e-11
MARGIN = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _gmm_from(F, quantile=0.6):
    """A mixture that splits the given features: nodes above the Q_Omega quantile form the
    viscous component, the rest the other one (means and covariances of each group)."""
    cut = np.quantile(F[2], quantile)
    hi, lo = F[:, F[2] > cut], F[:, F[2] <= cut]
    covs = []
    for grp in (lo, hi):
        C = np.cov(grp)
        covs.append(C + 1e-3 * np.diag(np.diag(C)) + 1e-30 * np.eye(3))
    return {"weights": np.array([lo.shape[1], hi.shape[1]], float), "means": np.stack([lo.mean(1), hi.mean(1)]),
            "covs": np.stack(covs), "viscous": 1}


def _gradient_scale(M, q, elements):
    return max(np.abs(rg.element_velocity_gradient(M, q, int(e))).max() for e in elements)


def _compare(S, M, q, gmm, elements=None, q_dev=None):
    import torch
    elements = np.arange(M.ne) if elements is None else np.asarray(elements)
    ref = rg.detect_regions(M, q, gmm, elements=elements)
    qd = to_dev(q) if q_dev is None else q_dev
    f, pb, ft = S.detect_regions(qd, gmm, features=True)
    torch.cuda.synchronize()
    f, pb, ft = f.cpu().numpy(), pb.cpu().numpy(), ft.cpu().numpy()
    idx = np.concatenate([np.arange(M.offsets[e], M.offsets[e + 1]) for e in elements])
    g = _gradient_scale(M, q, elements)
    for i, scale in ((0, g * g), (1, g ** 3), (2, g * g)):
        err = np.abs(ft[i, idx] - ref["features"][i]).max()
        assert err <= FEAT_TOL * max(scale, 1e-300), (i, err, scale)
    assert np.abs(ft[3, idx] - ref["p_v"]).max() <= PROB_TOL
    assert np.abs(pb[:, elements] - ref["pbar"]).max() <= PROB_TOL
    clear = np.abs(ref["pbar"][0] - ref["pbar"][1]) > MARGIN
    np.testing.assert_array_equal(f[elements][clear], ref["flags"][clear])
    assert set(np.unique(f)) <= {0, 1}
    return f, pb, ref


def _case_wake():
    return small_mixed(wl.wake_16x16x16_n4(n=8, order=4), seed=51, orders=(2, 5))


def _case_curved_mixed_orders():
    return small_mixed(wl.padapt_32x32x32(n=6), seed=52, orders=(2, 7))


def _case_rotated_all_orders():
    w = wl.tgv_4x4x4_n3(n_elem_dir=5, order=3)
    mesh, _ = wl.rotate_elements(w.mesh, 23)
    return small_mixed(dataclasses.replace(w, mesh=mesh), seed=53, orders=(1, 7))


def _case_channel():
    return small_mixed(wl.channel_walls(n=4, wall=3), seed=54, orders=(2, 6))


@pytest.mark.parametrize("make", [_case_wake, _case_curved_mixed_orders, _case_rotated_all_orders, _case_channel])
def test_detection_matches_the_oracle(make):
    w = make()
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    F = rg.detect_regions(M, q, {"weights": [1, 1], "means": np.zeros((2, 3)), "covs": np.stack([np.eye(3)] * 2),
                                 "viscous": 1})["features"]
    gmm = _gmm_from(F)
    S = gpu_solver(w)
    f, pb, ref = _compare(S, M, q, gmm)
    # a meaningful split: both regions present, and memberships strictly inside (0, 1) somewhere
    assert 0 < ref["flags"].sum() < w.n_elem
    assert np.any((ref["p_v"] > 1e-3) & (ref["p_v"] < 1 - 1e-3))
    # the flags feed the solver: set them and compare a residual with the oracle's
    S.set_flags(f)
    w2 = dataclasses.replace(w, flags=f)
    M2 = oracle_mesh(w2)
    R = S.residual(to_dev(q)).cpu().numpy()
    R_ref = M2.residual(q)
    assert np.sqrt(((R - R_ref) ** 2).sum() / (R_ref ** 2).sum()) <= 1e-12


def test_viscous_index_and_fp32_context():
    # the same mixture with its components listed the other way round gives the same answer,
    # and a reduced-precision context still detects in FP64
    w = _case_wake()
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    F = rg.detect_regions(M, q, {"weights": [1, 1], "means": np.zeros((2, 3)), "covs": np.stack([np.eye(3)] * 2),
                                 "viscous": 1})["features"]
    g = _gmm_from(F, quantile=0.5)
    swapped = {"weights": g["weights"][::-1].copy(), "means": g["means"][::-1].copy(), "covs": g["covs"][::-1].copy(),
               "viscous": 0}
    S = gpu_solver(w, precision=1)
    f1, pb1, _ = _compare(S, M, q, g)
    f2, pb2, _ = _compare(S, M, q, swapped)
    np.testing.assert_array_equal(f1, f2)
    assert np.abs(pb1 - pb2).max() <= PROB_TOL


def test_degenerate_states_and_ties():
    import torch
    w = _case_rotated_all_orders()
    M = oracle_mesh(w)
    S = gpu_solver(w)
    # a uniform flow: zero gradient, zero features, the same memberships everywhere
    q = np.zeros((4, M.total))
    q[1], q[2], q[3] = 1.0, -0.5, 0.25
    g = {"weights": [0.7, 0.3], "means": [[0.1, 0, 0.1], [-1, 0.1, 1]], "covs": np.stack([np.eye(3)] * 2),
         "viscous": 1}
    f, pb, ft = S.detect_regions(to_dev(q), g, features=True)
    torch.cuda.synchronize()
    # D annihilates constants up to rounding: gradients ~1e-15, features ~1e-30
    assert torch.abs(ft[:3]).max().item() <= 1e-26
    pv0, pi0 = rg.memberships(np.zeros((3, 1)), g)
    assert np.abs(ft[3].cpu().numpy() - pv0[0]).max() <= PROB_TOL
    assert np.abs(pb[0].cpu().numpy() - pv0[0]).max() <= PROB_TOL
    assert np.abs(pb[1].cpu().numpy() - pi0[0]).max() <= PROB_TOL
    assert torch.all(f == (1 if pv0[0] >= pi0[0] else 0))
    # identical components with equal weights: every mean is exactly 1/2, a tie, viscous
    tie = {"weights": [2.0, 2.0], "means": [[0.3, 0.1, 0.2]] * 2, "covs": np.stack([np.diag([1.0, 2.0, 3.0])] * 2),
           "viscous": 0}
    q = oracle_state(w, M)
    f, pb, _ = S.detect_regions(to_dev(q), tie)
    assert torch.all(pb == 0.5) and torch.all(f == 1)


def test_only_the_requested_outputs_are_written():
    import torch
    from paper_2403_05463_gb300 import dg
    w = _case_wake()
    M = oracle_mesh(w)
    q = to_dev(oracle_state(w, M))
    S = gpu_solver(w)
    g = dg.make_gmm([1, 1], [[0, 0, 0], [-0.1, 0, 0.1]], [np.eye(3)] * 2, 1)
    f, pb, ft = S.detect_regions(q, g, flags=True, pbar=False, features=False)
    assert pb is None and ft is None and f.shape == (w.n_elem,)
    f2, pb2, _ = S.detect_regions(q, g, flags=False, pbar=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(f.cpu().numpy(), (pb2[0] >= pb2[1]).to(torch.uint8).cpu().numpy())


@pytest.mark.parametrize("bad", ["not_spd", "not_symmetric", "weight", "viscous", "precision", "no_output"])
def test_bad_arguments_are_rejected(bad):
    import torch
    from paper_2403_05463_gb300 import dg
    w = _case_wake()
    S = gpu_solver(w)
    q = torch.zeros((4, S.total_nodes), dtype=torch.float64, device="cuda")
    covs = [np.eye(3), np.eye(3)]
    weights, viscous = [1.0, 1.0], 1
    if bad == "not_spd":
        covs[1] = np.diag([1.0, -1.0, 1.0])
    if bad == "not_symmetric":
        covs[0] = np.array([[1.0, 0.2, 0], [0, 1, 0], [0, 0, 1]])
    if bad == "weight":
        weights = [0.0, 1.0]
    if bad == "viscous":
        viscous = 2
    g = dg.make_gmm(weights, np.zeros((2, 3)), covs, viscous)
    if bad == "precision":
        g.precision = 2
    with pytest.raises(dg.DGError) as ei:
        if bad == "no_output":
            S.detect_regions(q, g, flags=False, pbar=False, features=False)
        else:
            S.detect_regions(q, g)
    assert dg.STATUS[ei.value.status] == "DG_ERR_ARG"


def test_full_size_sampled():
    """The 64^3 stretched mixed mesh at N = 4 (the benchmark's configuration), whole mesh on the
    GPU, a sample of elements on the oracle."""
    import torch
    from test_gpu_parity import _fourier_torch
    w = wl.mixed_64x64x64_n4()
    M = oracle_mesh(w)
    xyz = torch.from_numpy(M.node_coords()).cuda()
    q = torch.zeros((4, M.total), dtype=torch.float64, device="cuda")
    q[1:] = _fourier_torch(w, xyz)
    q[1] += 1.0
    del xyz
    qh = q.cpu().numpy()
    rng = np.random.default_rng(1)
    sel = np.concatenate([rng.choice(w.n_elem, 60, replace=False), [0, w.n_elem - 1]])
    F = rg.detect_regions(M, qh, {"weights": [1, 1], "means": np.zeros((2, 3)), "covs": np.stack([np.eye(3)] * 2),
                                  "viscous": 1}, elements=sel)["features"]
    gmm = _gmm_from(F, quantile=0.7)
    S = gpu_solver(w)
    f, pb, ref = _compare(S, M, qh, gmm, elements=sel, q_dev=q)
    assert 0 < f.sum() < w.n_elem


# FP32 pass (gmm precision 1): the gradient from the velocity rounded to FP32 carries ~1e-7 of
# |u| times ||D|| ~ 40, the features ~1e-6 of their scale, and the memberships that times the
# mixture's |d a / d x| (~1/sigma, up to ~100 here); the bounds below leave a factor ~10.
FP32_PROB_TOL = 2e-3
FP32_MARGIN = 1e-2


@pytest.mark.parametrize("make", [_case_wake, _case_curved_mixed_orders, _case_rotated_all_orders])
def test_fp32_detection_within_its_error(make):
    import json
    import os
    import torch
    w = make()
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    F = rg.detect_regions(M, q, {"weights": [1, 1], "means": np.zeros((2, 3)), "covs": np.stack([np.eye(3)] * 2),
                                 "viscous": 1})["features"]
    gmm = _gmm_from(F)
    ref = rg.detect_regions(M, q, gmm)
    S = gpu_solver(w, precision=1)
    f, pb, ft = S.detect_regions(to_dev(q), gmm, features=True, precision=1)
    torch.cuda.synchronize()
    f, pb, ft = f.cpu().numpy(), pb.cpu().numpy(), ft.cpu().numpy()
    g = _gradient_scale(M, q, range(M.ne))
    feat_err = max(np.abs(ft[i] - ref["features"][i]).max() / s for i, s in ((0, g * g), (1, g ** 3), (2, g * g)))
    p_err = np.abs(ft[3] - ref["p_v"]).max()
    pbar_err = np.abs(pb - ref["pbar"]).max()
    clear = np.abs(ref["pbar"][0] - ref["pbar"][1]) > FP32_MARGIN
    np.testing.assert_array_equal(f[clear], ref["flags"][clear])
    agree = float((f == ref["flags"]).mean())
    rec = {"case": "detect_fp32_" + w.name, "feature_rel": feat_err, "p_v_abs": float(p_err),
           "pbar_abs": float(pbar_err), "flags_agree": agree}
    print(rec)
    if os.environ.get("DG_PRECISION_LOG"):
        with open(os.environ["DG_PRECISION_LOG"], "a") as fh:
            fh.write(json.dumps(rec) + "\n")
    assert feat_err <= 1e-4, feat_err
    assert p_err <= FP32_PROB_TOL and pbar_err <= FP32_PROB_TOL, (p_err, pbar_err)


def test_detect_then_adapt_then_step():
    """The hybrid p-adapted workflow (Sec. 2.1 then Sec. 3.2), all through the C ABI: detect the
    regions on the current state, flag them, give the viscous region order P_v and the rest
    P_i, re-project the state onto the new orders, take RK steps; the oracle runs the same
    sequence from the same inputs (its own detection, projection and steps)."""
    import torch
    from oracle import oracle as orc
    w = wl.padapt_32x32x32(n=5)  # curved, degree-2 geometry, NS shear layer
    w = dataclasses.replace(w, orders=np.full(w.n_elem, 3, np.int8), flags=np.zeros(w.n_elem, np.uint8))
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    F = rg.detect_regions(M, q, {"weights": [1, 1], "means": np.zeros((2, 3)), "covs": np.stack([np.eye(3)] * 2),
                                 "viscous": 1})["features"]
    gmm = _gmm_from(F, quantile=0.7)
    # GPU: detect, flag, adapt, project, step
    S = gpu_solver(w)
    qd = to_dev(q)
    f, _, _ = S.detect_regions(qd, gmm, pbar=False)
    flags = f.cpu().numpy()
    orders = np.where(flags == 1, 5, 2).astype(np.int8)
    S.set_flags(flags)
    S.set_orders(orders)
    qd = S.project_state(qd)
    gd = torch.zeros_like(qd)
    S.rk_step(qd, gd, 1e-4, 3)
    # oracle: the same sequence (flags must agree outside near-ties; here every decision is clear)
    ref = rg.detect_regions(M, q, gmm)
    assert np.all(np.abs(ref["pbar"][0] - ref["pbar"][1]) > MARGIN)
    np.testing.assert_array_equal(flags, ref["flags"])
    assert 0 < flags.sum() < w.n_elem
    q2 = orc.project_state(w.orders, orders, q)
    w2 = dataclasses.replace(w, orders=orders, flags=flags)
    M2 = oracle_mesh(w2)
    g2 = np.zeros_like(q2)
    M2.rk_step(q2, g2, 1e-4, 3)
    got = qd.cpu().numpy()
    assert got.shape == q2.shape
    err = np.sqrt(((got - q2) ** 2).sum() / (q2 ** 2).sum())
    assert err <= 1e-12, err
