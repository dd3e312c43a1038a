"""Gauss-Legendre element nodes (dg_params.nodes = 1, App. B's quadrature) on the GPU, through the
C ABI, against the oracle on the same node set: node coordinates, residuals, RK steps and
conservation sums at the FP64 tolerance 1e-12 (relative L2) on box, re-oriented curved and every
order 1..7, mixed flags, Roe/LLF, Smagorinsky/Vreman, both mixed-face choices, inflow/outflow and
wall boundaries, p-nonconforming faces (mortars between Gauss point sets, orders 1..7), order and
node-set changes on a live context; the state re-projection and the allocation-free sums; the
region detection on the Gauss points; plus what the node set refuses."""
import dataclasses

import numpy as np
import pytest

from helpers import rel_l2, to_dev
from oracle import oracle as orc
from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle(w, params):
    m = w.mesh
    return orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, orc.params(**params), m.bc_tag)


def _solver(w, params):
    from paper_2403_05463_gb300 import dg
    return dg.Solver.from_workload(w, precision=0, params=dict(params))


def _box(order, n=4, seed=0):
    w = wl.tgv_4x4x4_n3(n_elem_dir=n, order=order)
    rng = np.random.default_rng(seed)
    return dataclasses.replace(w, flags=(rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8))


def _curved(order, seed):
    w = wl.padapt_32x32x32(n=4, amp=0.05)
    mesh, _ = wl.rotate_elements(w.mesh, seed)
    rng = np.random.default_rng(seed)
    flags = (rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8)
    return dataclasses.replace(w, mesh=mesh, orders=np.full(w.n_elem, order, np.int8), flags=flags)


def _gl(w, **kw):
    return dict(w.params, nodes=1, **kw)


CASES = [
    ("box_n4", lambda: _box(4), dict(nu=1e-2)),
    ("box_n3_vreman_llf_onesided", lambda: _box(3, seed=1), dict(nu=1e-2, closure=1, riemann=1, mixed_face=1)),
    ("curved_n3", lambda: _curved(3, 61), dict(nu=1e-2)),
    ("curved_n5", lambda: _curved(5, 62), dict(nu=1e-2, closure=1)),
]


@pytest.mark.parametrize("name,make,extra", CASES, ids=[c[0] for c in CASES])
def test_residual_matches_the_oracle(name, make, extra):
    w = make()
    p = _gl(w, **extra)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    R_ref = M.residual(q)
    S = _solver(w, p)
    np.testing.assert_allclose(S.node_coords().cpu().numpy(), M.node_coords(), atol=1e-13)
    R = S.residual(to_dev(q)).cpu().numpy()
    err = rel_l2(R, R_ref)
    assert err <= TOL, err
    assert np.abs(R - R_ref).max() <= 10 * TOL * np.abs(R_ref).max()


@pytest.mark.parametrize("order", [1, 2, 6, 7])
def test_every_order(order):
    w = _box(1, n=5) if order == 1 else _curved(order, 70 + order)
    p = _gl(w, nu=1e-2)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    R = _solver(w, p).residual(to_dev(q)).cpu().numpy()
    assert rel_l2(R, M.residual(q)) <= TOL


def test_rk_steps_and_conservation():
    w = _curved(3, 80)
    p = _gl(w, nu=1e-2)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    g = np.zeros_like(q)
    S = _solver(w, p)
    qd, gd = to_dev(q), to_dev(g)
    S.rk_step(qd, gd, 1e-3, 5)
    M.rk_step(q, g, 1e-3, 5)
    assert rel_l2(qd.cpu().numpy(), q) <= TOL
    R = S.residual(qd)
    sums = S.conservation(R)
    scale = np.abs(R.cpu().numpy()).max()
    assert np.all(np.abs(sums) <= 1e-11 * scale), sums
    np.testing.assert_allclose(sums, M.conservation(R.cpu().numpy()), atol=1e-11 * scale)


@pytest.mark.parametrize("make", [lambda: wl.wake_16x16x16_n4(n=6, order=4),
                                  lambda: wl.channel_walls(n=4, wall=3), lambda: wl.channel_walls(n=4, wall=4)],
                         ids=["wake_inflow_outflow", "channel_noslip", "channel_slip"])
def test_boundary_faces(make):
    # inflow/outflow ghosts and no-slip/free-slip mirror walls on Gauss points, mixed flags
    w = make()
    rng = np.random.default_rng(5)
    w = dataclasses.replace(w, flags=(rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8))
    p = _gl(w, nu=1e-2)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    R = _solver(w, p).residual(to_dev(q)).cpu().numpy()
    assert rel_l2(R, M.residual(q)) <= TOL


def test_what_gauss_legendre_refuses():
    import torch
    from paper_2403_05463_gb300 import dg
    w = _box(3)
    p = _gl(w)
    S = _solver(w, p)
    for bad, prec in ((dict(split=1), 0), ({}, 1)):
        with pytest.raises(dg.DGError):
            S.set_params(dict(p, **bad), precision=prec)
    S.set_params(p, precision=0)


def test_state_reprojection_and_allocation_free_sums_on_gauss_points():
    """dg_project_state after two re-assignments of orders on a curved mesh (interpolation
    onto the new Gauss points, L2 projection where the order drops) against the oracle's, then
    the residual on the re-laid-out state, and dg_conservation_noalloc with the Gauss weights."""
    import torch
    w = _mixed(_curved(3, 97), 97, 2, 7)
    p = _gl(w, nu=1e-2)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    S = _solver(w, p)
    rng = np.random.default_rng(98)
    o_prev, q_prev, qd = w.orders.copy(), q, to_dev(q)
    for _ in range(2):
        o_new = rng.integers(2, 8, size=w.n_elem).astype(np.int8)
        S.set_orders(o_new)
        qd = S.project_state(qd)
        torch.cuda.synchronize()
        ref = orc.project_state(o_prev, o_new, q_prev, nodes=1)
        assert np.abs(qd.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
        o_prev, q_prev = o_new, ref
    w2 = dataclasses.replace(w, orders=o_prev)
    M2 = _oracle(w2, p)
    R = S.residual(qd)
    assert rel_l2(R.cpu().numpy(), M2.residual(q_prev)) <= TOL
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    S.conservation_noalloc(R, out)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), S.conservation(R), rtol=0,
                               atol=1e-13 * np.abs(R.cpu().numpy()).max())


def _mixed(w, seed, lo, hi):
    rng = np.random.default_rng(seed)
    return dataclasses.replace(w, orders=rng.integers(lo, hi + 1, size=w.n_elem).astype(np.int8))


MORTAR_CASES = [
    ("box_orders_1_7", lambda: _mixed(_box(3, n=5, seed=3), 90, 1, 7), dict(nu=1e-2)),
    ("curved_orders_2_6_vreman_llf", lambda: _mixed(_curved(3, 91), 91, 2, 6), dict(nu=1e-2, closure=1, riemann=1)),
    ("curved_orders_2_5_onesided", lambda: _mixed(_curved(3, 92), 92, 2, 5), dict(nu=1e-2, mixed_face=1)),
    ("channel_noslip_orders_2_5", lambda: _mixed(wl.channel_walls(n=4, wall=3), 93, 2, 5), dict(nu=1e-2)),
    ("wake_orders_2_5", lambda: _mixed(wl.wake_16x16x16_n4(n=6, order=4), 94, 2, 5), dict(nu=1e-2)),
]


@pytest.mark.parametrize("name,make,extra", MORTAR_CASES, ids=[c[0] for c in MORTAR_CASES])
def test_p_nonconforming_faces(name, make, extra):
    """Mortars between Gauss point sets (Sec. 3.2 on App. B's nodes): the residual on meshes
    whose neighbouring elements differ in order, mixed flags, against the oracle at 1e-12."""
    w = make()
    rng = np.random.default_rng(7)
    w = dataclasses.replace(w, flags=(rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8))
    p = _gl(w, **extra)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    R = _solver(w, p).residual(to_dev(q)).cpu().numpy()
    assert rel_l2(R, M.residual(q)) <= TOL


def test_mortar_rk_steps_conservation_and_order_changes():
    # RK steps on a mixed-order curved mesh, the conservation sums, then a change of orders
    # through dg_set_orders and a change of node set through dg_set_params on the same context
    w = _mixed(_curved(3, 95), 95, 2, 6)
    p = _gl(w, nu=1e-2)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    g = np.zeros_like(q)
    S = _solver(w, p)
    qd, gd = to_dev(q), to_dev(g)
    S.rk_step(qd, gd, 1e-3, 4)
    M.rk_step(q, g, 1e-3, 4)
    assert rel_l2(qd.cpu().numpy(), q) <= TOL
    R = S.residual(qd)
    sums = S.conservation(R)
    scale = np.abs(R.cpu().numpy()).max()
    assert np.all(np.abs(sums) <= 1e-11 * scale), sums
    w2 = _mixed(w, 96, 2, 7)  # the degree-2 geometry needs N >= 2
    S.set_orders(w2.orders)
    M2 = _oracle(w2, p)
    q2 = w2.state(M2.node_coords())
    np.testing.assert_allclose(S.node_coords().cpu().numpy(), M2.node_coords(), atol=1e-13)
    assert rel_l2(S.residual(to_dev(q2)).cpu().numpy(), M2.residual(q2)) <= TOL
    # back to Gauss-Lobatto nodes, then Gauss points again: the nodes, metric terms and tables
    # follow the node set
    p0 = dict(p, nodes=0)
    S.set_params(p0, precision=0)
    M0 = _oracle(w2, p0)
    q0 = w2.state(M0.node_coords())
    np.testing.assert_allclose(S.node_coords().cpu().numpy(), M0.node_coords(), atol=1e-13)
    assert rel_l2(S.residual(to_dev(q0)).cpu().numpy(), M0.residual(q0)) <= TOL
    S.set_params(p, precision=0)
    assert rel_l2(S.residual(to_dev(q2)).cpu().numpy(), M2.residual(q2)) <= TOL


@pytest.mark.parametrize("make,precision", [(lambda: _box(3, n=5, seed=2), 0), (lambda: _curved(5, 63), 0),
                                            (lambda: _curved(4, 64), 1)], ids=["box_n3", "curved_n5", "curved_n4_fp32"])
def test_region_detection_on_gauss_points(make, precision):
    """Sec. 2.1's detection on the Gauss-Legendre points the paper clusters: features, node
    memberships, element means and flags against the oracle on the same node set (FP64 at the
    region tests' bars; FP32 within its own error), and the flags fed back into the residual."""
    import torch
    from oracle import regions as rg
    from test_gpu_regions import FP32_MARGIN, FP32_PROB_TOL, _gmm_from, _gradient_scale
    w = make()
    p = _gl(w, nu=1e-2)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    F = rg.detect_regions(M, q, {"weights": [1, 1], "means": np.zeros((2, 3)), "covs": np.stack([np.eye(3)] * 2),
                                 "viscous": 1})["features"]
    gmm = _gmm_from(F)
    ref = rg.detect_regions(M, q, gmm)
    assert 0 < ref["flags"].sum() < w.n_elem
    S = _solver(w, p)
    f, pb, ft = S.detect_regions(to_dev(q), gmm, features=True, precision=precision)
    torch.cuda.synchronize()
    f, pb, ft = f.cpu().numpy(), pb.cpu().numpy(), ft.cpu().numpy()
    g = _gradient_scale(M, q, range(M.ne))
    # the FP32 bounds are those of the Lobatto FP32 detection test
    feat_tol, prob_tol, margin = (1e-12, 1e-11, 1e-9) if precision == 0 else (1e-4, FP32_PROB_TOL, FP32_MARGIN)
    for i, scale in ((0, g * g), (1, g ** 3), (2, g * g)):
        assert np.abs(ft[i] - ref["features"][i]).max() <= feat_tol * scale, i
    assert np.abs(ft[3] - ref["p_v"]).max() <= prob_tol
    assert np.abs(pb - ref["pbar"]).max() <= prob_tol
    clear = np.abs(ref["pbar"][0] - ref["pbar"][1]) > margin
    np.testing.assert_array_equal(f[clear], ref["flags"][clear])
    S.set_flags(f)
    R = S.residual(to_dev(q)).cpu().numpy()
    R_ref = _oracle(dataclasses.replace(w, flags=f), p).residual(q)
    assert rel_l2(R, R_ref) <= TOL


def test_a_32cube_case_sampled():
    """tgv 32^3 at N = 5 on Gauss-Legendre nodes (4.4 M nodes), 30% NS: the whole mesh on the
    GPU, a sample of elements on the oracle."""
    w = wl.tgv_32x32x32_n5()
    p = _gl(w, nu=1e-3)
    M = _oracle(w, p)
    q = w.state(M.node_coords())
    R = _solver(w, p).residual(to_dev(q)).cpu().numpy()
    rng = np.random.default_rng(3)
    ns, eu = np.flatnonzero(w.flags), np.flatnonzero(w.flags == 0)
    sel = np.concatenate([rng.choice(ns, 20, replace=False), rng.choice(eu, 20, replace=False), [0, w.n_elem - 1]])
    idx = np.concatenate([np.arange(M.offsets[e], M.offsets[e + 1]) for e in sel])
    R_ref = np.zeros_like(q)
    M.residual(q, sel=sel, out=R_ref)
    assert rel_l2(R[:, idx], R_ref[:, idx]) <= TOL
