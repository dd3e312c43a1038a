"""Compressible form (App. A, dg_params.model = 1) on the GPU, through the C ABI, against the FP64
oracle's compressible entry points: residuals, RK steps and conservation sums at the FP64
tolerance 1e-12 (relative L2), on box, re-oriented curved and every order 1..7, mixed flags,
Roe/LLF, Vreman/Smagorinsky, both mixed-face choices, far-field inflow / pressure outflow and
adiabatic no-slip/free-slip walls, p-nonconforming faces (orders 1..7), and all of these on the
Gauss-Legendre nodes too; plus what the build rejects."""
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


def _oracle(w, params=None):
    p = dict(params or w.params)
    p.pop("model", None)
    m = w.mesh
    return orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, orc.params(**p), m.bc_tag)


def _solver(w, params=None):
    from paper_2403_05463_gb300 import dg
    return dg.Solver.from_workload(w, precision=0, params=params)


def _state(w, M):
    return wl.cns_state(M.node_coords(), w.seed, period=2 * np.pi if "tgv" in w.name else 1.0)


def _curved_small(order, seed, flags_p=0.5):
    w = wl.padapt_32x32x32(n=4, amp=0.05)
    mesh, _ = wl.rotate_elements(w.mesh, seed)
    rng = np.random.default_rng(seed)
    flags = (rng.uniform(size=w.n_elem) < flags_p).astype(np.uint8)
    params = dict(wl.cns_tgv().params)
    return dataclasses.replace(w, mesh=mesh, orders=np.full(w.n_elem, order, np.int8), flags=flags, params=params,
                               name=f"cns_padapt_4x4x4_n{order}")


def _box(order, n=4):
    return wl.cns_tgv(n=n, order=order)


CASES = [
    ("box_n4_vreman_roe", lambda: _box(4), {}),
    ("box_n3_smagorinsky_llf_onesided", lambda: _box(3), dict(closure=0, riemann=1, mixed_face=1)),
    ("curved_n3", lambda: _curved_small(3, 31), {}),
    ("curved_n5_all_ns", lambda: dataclasses.replace(_curved_small(5, 32), flags=np.ones(64, np.uint8)), {}),
    ("curved_tgv_n4", lambda: wl.cns_tgv(n=4, order=4, curved=True), dict(nu=1e-2)),
]


@pytest.mark.parametrize("name,make,extra", CASES, ids=[c[0] for c in CASES])
def test_residual_matches_the_oracle(name, make, extra):
    w = make()
    p = dict(w.params, **extra)
    M = _oracle(w, p)
    u = _state(w, M)
    R_ref = M.cns_residual(u)
    S = _solver(w, p)
    assert S.nvar == 5 and S.total_nodes == M.total
    R = S.residual(to_dev(u)).cpu().numpy()
    err = rel_l2(R, R_ref)
    assert err <= TOL, err
    assert np.abs(R - R_ref).max() <= 10 * TOL * np.abs(R_ref).max()


@pytest.mark.parametrize("order", [1, 2, 6, 7])
def test_every_order(order):
    w = _curved_small(order, 40 + order) if order >= 2 else _box(1, n=5)
    M = _oracle(w)
    u = _state(w, M)
    R = _solver(w).residual(to_dev(u)).cpu().numpy()
    assert rel_l2(R, M.cns_residual(u)) <= TOL


def test_rk_steps_and_conservation():
    w = _curved_small(3, 50)
    p = dict(w.params, nu=5e-3)
    M = _oracle(w, p)
    u = _state(w, M)
    g = np.zeros_like(u)
    S = _solver(w, p)
    ud, gd = to_dev(u), to_dev(g)
    S.rk_step(ud, gd, 1e-3, 5)
    M.cns_rk_step(u, g, 1e-3, 5)
    assert rel_l2(ud.cpu().numpy(), u) <= TOL
    assert rel_l2(gd.cpu().numpy(), g) <= 1e-11  # g ~ dt R: the same relative bar, rounding of the increments
    R = S.residual(ud)
    sums = S.conservation(R)
    assert sums.shape == (5,)
    ref = M.cns_conservation(R.cpu().numpy())
    scale = np.abs(R.cpu().numpy()).max()
    assert np.all(np.abs(sums) <= 1e-11 * scale) and np.all(np.abs(ref) <= 1e-11 * scale)


def test_model_switch_on_an_existing_context():
    import torch
    w = _box(3)
    p0 = dict(w.params, model=0)
    S = _solver(w, p0)
    assert S.nvar == 4
    S.set_params(dict(w.params))
    assert S.nvar == 5
    M = _oracle(w)
    u = _state(w, M)
    R = S.residual(to_dev(u)).cpu().numpy()
    assert rel_l2(R, M.cns_residual(u)) <= TOL
    with pytest.raises(ValueError):
        S.residual(torch.zeros((4, S.total_nodes), dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("wall", [3, 4])
def test_adiabatic_walls(wall):
    # the wavy degree-2 channel between walls, re-oriented elements, mixed flags, one order
    w = wl.channel_walls(n=4, wall=wall)
    mesh, _ = wl.rotate_elements(w.mesh, 90 + wall)
    rng = np.random.default_rng(wall)
    w = dataclasses.replace(w, mesh=mesh, flags=(rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8),
                            params=dict(wl.cns_tgv().params, nu=1e-2))
    M = _oracle(w)
    u = wl.cns_state(M.node_coords(), w.seed, period=2 * np.pi)
    R_ref = M.cns_residual(u)
    S = _solver(w)
    R = S.residual(to_dev(u)).cpu().numpy()
    assert rel_l2(R, R_ref) <= TOL, rel_l2(R, R_ref)
    sums = S.conservation(to_dev(R))
    scale = np.abs(R).max()
    assert abs(sums[0]) <= 1e-11 * scale and abs(sums[4]) <= 1e-11 * scale, sums  # walls pass no mass, energy


def test_inflow_outflow():
    # the wake box: far-field inflow at x = 0, pressure outflow at x = 8, periodic in y and z,
    # mixed flags
    w = wl.wake_16x16x16_n4(n=5, order=3)
    rng = np.random.default_rng(7)
    w = dataclasses.replace(w, flags=(rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8),
                            params=dict(wl.cns_tgv().params, nu=1e-2, inflow=(1.05, 0.6, 0.0, 0.05), p_inf=16.0))
    M = _oracle(w)
    u = wl.cns_state(M.node_coords(), w.seed, period=4.0)
    R_ref = M.cns_residual(u)
    R = _solver(w).residual(to_dev(u)).cpu().numpy()
    assert rel_l2(R, R_ref) <= TOL, rel_l2(R, R_ref)


def test_what_the_compressible_build_rejects():
    import torch
    from paper_2403_05463_gb300 import dg
    p = dict(wl.cns_tgv().params)
    # inflow/outflow faces without a far field
    wake = wl.wake_16x16x16_n4(n=3, order=2)
    with pytest.raises(dg.DGError) as ei:
        dg.Solver.from_workload(wake, params=p)
    assert dg.STATUS[ei.value.status] == "DG_ERR_ARG"
    w = _box(3)
    S = _solver(w)
    # reduced precision, split form, bad gas constants
    for bad in (dict(precision=1), dict(split=1), dict(gamma=1.0)):
        with pytest.raises(dg.DGError):
            S.set_params(dict(p, **{k: v for k, v in bad.items() if k != "precision"}),
                         precision=bad.get("precision", 0))
    S.set_params(p, precision=0)
    u = torch.ones((5, S.total_nodes), dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError):
        S.detect_regions(u, {"weights": [1, 1], "means": np.zeros((2, 3)), "covs": [np.eye(3)] * 2, "viscous": 1})
    with pytest.raises(dg.DGError):
        S.conservation_noalloc(u, torch.zeros(5, dtype=torch.float64, device="cuda"))


def _mixed(w, seed, lo, hi):
    rng = np.random.default_rng(seed)
    return dataclasses.replace(w, orders=rng.integers(lo, hi + 1, size=w.n_elem).astype(np.int8))


MORTAR_CASES = [
    ("box_orders_1_7_vreman_roe", lambda: _mixed(_box(3, n=5), 60, 1, 7), {}),
    ("curved_orders_2_6_smagorinsky_llf_onesided", lambda: _mixed(_curved_small(3, 61), 61, 2, 6),
     dict(closure=0, riemann=1, mixed_face=1)),
    ("curved_orders_2_5_all_ns", lambda: dataclasses.replace(_mixed(_curved_small(3, 62), 62, 2, 5),
                                                              flags=np.ones(64, np.uint8)), dict(nu=1e-2)),
]


@pytest.mark.parametrize("name,make,extra", MORTAR_CASES, ids=[c[0] for c in MORTAR_CASES])
def test_p_nonconforming_faces(name, make, extra):
    """Five-variable mortars (Sec. 3.2): interpolated states and viscous traces, Roe/LLF and the
    BR1 average of (v, T) on the mortar, L2 projection back, against the oracle at 1e-12."""
    w = make()
    p = dict(w.params, **extra)
    M = _oracle(w, p)
    u = _state(w, M)
    R = _solver(w, p).residual(to_dev(u)).cpu().numpy()
    assert rel_l2(R, M.cns_residual(u)) <= TOL


def test_mortars_with_walls_rk_steps_and_order_changes():
    # the wall channel with orders 2..5, RK steps against the oracle's, conservation of mass and
    # energy through the walls, then new orders on the same context
    w = wl.channel_walls(n=4, wall=3)
    rng = np.random.default_rng(63)
    w = dataclasses.replace(w, flags=(rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8),
                            orders=rng.integers(2, 6, size=w.n_elem).astype(np.int8),
                            params=dict(wl.cns_tgv().params, nu=1e-2))
    M = _oracle(w)
    u = wl.cns_state(M.node_coords(), w.seed, period=2 * np.pi)
    g = np.zeros_like(u)
    S = _solver(w)
    ud, gd = to_dev(u), to_dev(g)
    S.rk_step(ud, gd, 1e-3, 3)
    M.cns_rk_step(u, g, 1e-3, 3)
    assert rel_l2(ud.cpu().numpy(), u) <= TOL
    R = S.residual(ud)
    sums = S.conservation(R)
    scale = np.abs(R.cpu().numpy()).max()
    assert abs(sums[0]) <= 1e-11 * scale and abs(sums[4]) <= 1e-11 * scale, sums
    w2 = dataclasses.replace(w, orders=rng.integers(2, 8, size=w.n_elem).astype(np.int8))
    S.set_orders(w2.orders)
    M2 = _oracle(w2)
    u2 = wl.cns_state(M2.node_coords(), w.seed, period=2 * np.pi)
    assert rel_l2(S.residual(to_dev(u2)).cpu().numpy(), M2.cns_residual(u2)) <= TOL


@pytest.mark.parametrize("nodes", [0, 1], ids=["lobatto", "legendre"])
def test_state_reprojection_after_order_changes(nodes):
    """dg_project_state on the five-plane compressible state (Sec. 3.2: restarting with
    re-assigned orders) after two re-assignments on a curved mesh, against the oracle's, then
    the residual on the re-laid-out state."""
    import torch
    w = _mixed(_curved_small(3, 75), 75, 2, 7)
    p = dict(w.params, nodes=nodes)
    M = _oracle(w, p)
    u = _state(w, M)
    S = _solver(w, p)
    rng = np.random.default_rng(76)
    o_prev, u_prev, ud = w.orders.copy(), u, to_dev(u)
    for _ in range(2):
        o_new = rng.integers(2, 8, size=w.n_elem).astype(np.int8)
        S.set_orders(o_new)
        ud = S.project_state(ud)
        torch.cuda.synchronize()
        ref = orc.project_state(o_prev, o_new, u_prev, nodes=nodes)
        assert ud.shape == ref.shape
        assert np.abs(ud.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
        o_prev, u_prev = o_new, ref
    M2 = _oracle(dataclasses.replace(w, orders=o_prev), p)
    assert rel_l2(S.residual(ud).cpu().numpy(), M2.cns_residual(u_prev)) <= TOL


GL_CASES = [
    ("box_n3", lambda: _box(3), {}),
    ("box_n1_llf_onesided", lambda: _box(1, n=5), dict(riemann=1, mixed_face=1, closure=0)),
    ("curved_n5", lambda: _curved_small(5, 70), {}),
    ("curved_n7_all_ns", lambda: dataclasses.replace(_curved_small(7, 71), flags=np.ones(64, np.uint8)), dict(nu=1e-2)),
    ("curved_orders_2_6_mortars", lambda: _mixed(_curved_small(3, 72), 72, 2, 6), {}),
    ("box_orders_1_7_mortars_smagorinsky", lambda: _mixed(_box(3, n=5), 73, 1, 7), dict(closure=0)),
]


@pytest.mark.parametrize("name,make,extra", GL_CASES, ids=[c[0] for c in GL_CASES])
def test_gauss_legendre_nodes(name, make, extra):
    """The compressible form on the Gauss-Legendre points (App. A on App. B's nodes): interpolated
    face states and viscous traces, l_i(+-1)/w_i lifting, Gauss-point mortars; against the oracle
    on the same node set at 1e-12."""
    w = make()
    p = dict(w.params, nodes=1, **extra)
    M = _oracle(w, p)
    u = _state(w, M)
    S = _solver(w, p)
    np.testing.assert_allclose(S.node_coords().cpu().numpy(), M.node_coords(), atol=1e-13)
    R = S.residual(to_dev(u)).cpu().numpy()
    assert rel_l2(R, M.cns_residual(u)) <= TOL


def test_gauss_legendre_boundaries_rk_steps_and_conservation():
    # walls (no-slip, free-slip) with mixed orders, the far-field wake box, then RK steps and the
    # conservation sums with the Gauss weights
    for wall in (3, 4):
        w = wl.channel_walls(n=4, wall=wall)
        rng = np.random.default_rng(80 + wall)
        w = dataclasses.replace(w, flags=(rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8),
                                orders=rng.integers(2, 6, size=w.n_elem).astype(np.int8),
                                params=dict(wl.cns_tgv().params, nu=1e-2, nodes=1))
        M = _oracle(w)
        u = wl.cns_state(M.node_coords(), w.seed, period=2 * np.pi)
        S = _solver(w)
        R = S.residual(to_dev(u)).cpu().numpy()
        assert rel_l2(R, M.cns_residual(u)) <= TOL, wall
        sums = S.conservation(to_dev(R))
        assert abs(sums[0]) <= 1e-11 * np.abs(R).max() and abs(sums[4]) <= 1e-11 * np.abs(R).max(), sums
    w = wl.wake_16x16x16_n4(n=5, order=3)
    rng = np.random.default_rng(82)
    w = dataclasses.replace(w, flags=(rng.uniform(size=w.n_elem) < 0.5).astype(np.uint8),
                            params=dict(wl.cns_tgv().params, nu=1e-2, inflow=(1.05, 0.6, 0.0, 0.05), p_inf=16.0,
                                        nodes=1))
    M = _oracle(w)
    u = wl.cns_state(M.node_coords(), w.seed, period=4.0)
    S = _solver(w)
    assert rel_l2(S.residual(to_dev(u)).cpu().numpy(), M.cns_residual(u)) <= TOL
    g = np.zeros_like(u)
    ud, gd = to_dev(u), to_dev(g)
    S.rk_step(ud, gd, 1e-3, 3)
    M.cns_rk_step(u, g, 1e-3, 3)
    assert rel_l2(ud.cpu().numpy(), u) <= TOL


@pytest.mark.parametrize("nodes", [0, 1], ids=["lobatto", "legendre"])
def test_a_32cube_case_sampled(nodes):
    """cns_tgv 32^3 at N = 4 (4.1 M nodes), 30% NS, the configuration the benchmark times on
    either node set: the whole mesh on the GPU, a sample of elements on the oracle."""
    import torch
    w = wl.cns_tgv(n=32, order=4)
    w = dataclasses.replace(w, params=dict(w.params, nodes=nodes))
    M = _oracle(w)
    u = _state(w, M)
    S = _solver(w)
    R = S.residual(to_dev(u)).cpu().numpy()
    rng = np.random.default_rng(2)
    ns, eu = np.flatnonzero(w.flags), np.flatnonzero(w.flags == 0)
    sel = np.concatenate([rng.choice(ns, 20, replace=False), rng.choice(eu, 20, replace=False), [0, w.n_elem - 1]])
    idx = np.concatenate([np.arange(M.offsets[e], M.offsets[e + 1]) for e in sel])
    R_ref = np.zeros_like(u)
    M.cns_residual(u, sel=sel, out=R_ref)
    assert rel_l2(R[:, idx], R_ref[:, idx]) <= TOL
    torch.cuda.synchronize()
