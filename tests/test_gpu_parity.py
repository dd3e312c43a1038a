"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

FP64 bar: relative L2 <= 1e-12 per residual (and after 10 RK3 steps on the Taylor-Green
workload), the tolerance the hot path is specified to; max-abs checked at 1e-11 of max |R|.
"""
import dataclasses

import numpy as np
import pytest

from helpers import gpu_solver, oracle_mesh, oracle_state, rel_l2, small_mixed, to_dev
from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _residual_pair(w, params=None, precision=0):
    M = oracle_mesh(w, params)
    q = oracle_state(w, M)
    R_ref = M.residual(q)
    S = gpu_solver(w, precision=precision, params=params)
    assert S.total_nodes == M.total
    np.testing.assert_array_equal(S.offsets, M.offsets)
    R = S.residual(to_dev(q)).cpu().numpy()
    return R, R_ref, M, S, q


def _assert_parity(R, R_ref, tol=TOL):
    err = rel_l2(R, R_ref)
    assert err <= tol, err
    assert np.abs(R - R_ref).max() <= 10 * tol * np.abs(R_ref).max()


def test_node_coordinates_match():
    w = small_mixed(wl.padapt_32x32x32(n=3), seed=1, orders=(2, 7))
    M = oracle_mesh(w)
    S = gpu_solver(w)
    np.testing.assert_allclose(S.node_coords().cpu().numpy(), M.node_coords(), atol=1e-13)


def test_tgv_4x4x4_n3_residual():
    R, R_ref, *_ = _residual_pair(wl.tgv_4x4x4_n3())
    _assert_parity(R, R_ref)


def test_tgv_4x4x4_n3_rk3_10_steps():
    w = wl.tgv_4x4x4_n3()
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    g = np.zeros_like(q)
    qd, gd = to_dev(q), to_dev(np.full_like(q, np.nan))  # g need not be initialised
    S = gpu_solver(w)
    S.rk_step(qd, gd, w.dt, w.steps)
    M.rk_step(q, g, w.dt, w.steps)
    assert rel_l2(qd.cpu().numpy(), q) <= TOL
    dq_gpu = qd.cpu().numpy() - oracle_state(w, M)
    dq_ref = q - oracle_state(w, M)
    assert rel_l2(dq_gpu, dq_ref) <= 1e-10  # the update itself, not only the state


def test_wake_16x16x16_n4_mixed_and_all_ns():
    w = wl.wake_16x16x16_n4()
    assert 0.10 < w.ns_fraction < 0.15
    R, R_ref, *_ = _residual_pair(w)
    _assert_parity(R, R_ref)
    w_ns = w.with_flags(np.ones(w.n_elem))
    R2, R2_ref, *_ = _residual_pair(w_ns)
    _assert_parity(R2, R2_ref)


@pytest.mark.parametrize("closure,riemann", [(0, 1), (1, 0), (1, 1)])
def test_variants_closure_and_flux(closure, riemann):
    w = small_mixed(wl.tgv_32x32x32_n5(n=5), seed=2)
    p = dict(w.params, closure=closure, riemann=riemann, nu=1e-3, cs=0.17, cv=0.3)
    R, R_ref, *_ = _residual_pair(w, params=p)
    _assert_parity(R, R_ref)


def test_tgv_slab_ragged_tail_n5():
    # 7^3 = 343 elements at N = 5 (one element per block) with a ragged 30% slab
    w = wl.tgv_32x32x32_n5(n=7)
    R, R_ref, *_ = _residual_pair(w)
    _assert_parity(R, R_ref)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6, 7])
def test_every_order_uniform(N):
    # 5^3 = 125 elements: ragged tails for every elements-per-block packing
    base = wl.tgv_4x4x4_n3(n_elem_dir=5, order=N)
    w = small_mixed(base, seed=10 + N)
    R, R_ref, *_ = _residual_pair(w, params=dict(w.params, nu=0.01))
    _assert_parity(R, R_ref)


def test_curved_mixed_orders_rotated_elements():
    w = wl.padapt_32x32x32(n=4)
    mesh, _ = wl.rotate_elements(w.mesh, 5)
    w = small_mixed(dataclasses.replace(w, mesh=mesh), seed=3, orders=(2, 7))
    R, R_ref, *_ = _residual_pair(w, params=dict(w.params, nu=1e-2))
    _assert_parity(R, R_ref)


def test_one_sided_mixed_face():
    # the one-sided Euler/NS face flux on a curved, rotated mesh with mortars (orders 2..6)
    # and on the wake box (inflow/outflow faces); it must differ from the default average
    w = wl.padapt_32x32x32(n=4)
    mesh, _ = wl.rotate_elements(w.mesh, 9)
    w = small_mixed(dataclasses.replace(w, mesh=mesh), seed=13, orders=(2, 6))
    p1 = dict(w.params, nu=1e-2, mixed_face=1)
    R, R_ref, M, S, q = _residual_pair(w, params=p1)
    _assert_parity(R, R_ref)
    R0 = oracle_mesh(w, dict(p1, mixed_face=0)).residual(q)
    assert rel_l2(R_ref, R0) > 1e-6
    ww = wl.wake_16x16x16_n4(n=8)
    R2, R2_ref, *_ = _residual_pair(ww, params=dict(ww.params, nu=1e-3, mixed_face=1))
    _assert_parity(R2, R2_ref)


@pytest.mark.parametrize("rotated", [False, True])
def test_kep_split_form(rotated):
    # the kinetic-energy-preserving split form: curved mesh with mortars (orders 2..6) and
    # mixed flags, optionally with every element re-oriented
    w = wl.padapt_32x32x32(n=4)
    if rotated:
        mesh, _ = wl.rotate_elements(w.mesh, 19)
        w = dataclasses.replace(w, mesh=mesh)
    w = small_mixed(w, seed=17, orders=(2, 6))
    p = dict(w.params, nu=1e-2, split=1)
    R, R_ref, M, S, q = _residual_pair(w, params=p)
    _assert_parity(R, R_ref)
    assert rel_l2(R_ref, oracle_mesh(w, dict(p, split=0)).residual(q)) > 1e-6  # differs from the standard form


def test_kep_box_and_rk_steps():
    ww = wl.wake_16x16x16_n4(n=8)
    R, R_ref, *_ = _residual_pair(ww, params=dict(ww.params, split=1))
    _assert_parity(R, R_ref)
    w = wl.tgv_4x4x4_n3()
    p = dict(w.params, split=1)
    M = oracle_mesh(w, p)
    q = oracle_state(w, M)
    q0 = q.copy()
    g = np.zeros_like(q)
    qd, gd = to_dev(q), to_dev(g)
    S = gpu_solver(w, params=p)
    S.rk_step(qd, gd, w.dt, w.steps)
    M.rk_step(q, g, w.dt, w.steps)
    assert rel_l2(qd.cpu().numpy() - q0, q - q0) <= 1e-10


def test_project_state_after_order_change():
    # dynamic p-adaptation: orders re-assigned twice on a curved mesh; the state follows
    from oracle import oracle as orc
    import torch
    w = small_mixed(wl.padapt_32x32x32(n=4), seed=21, orders=(2, 7))
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    S = gpu_solver(w)
    rng = np.random.default_rng(22)
    o_prev, q_prev = w.orders.copy(), q
    qd = to_dev(q)
    for _ in range(2):
        o_new = rng.integers(2, 8, size=w.n_elem).astype(np.int8)
        S.set_orders(o_new)
        qd = S.project_state(qd)
        torch.cuda.synchronize()
        ref = orc.project_state(o_prev, o_new, q_prev)
        got = qd.cpu().numpy()
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        o_prev, q_prev = o_new, ref
    # and the residual runs on the re-laid-out state
    R = S.residual(qd).cpu().numpy()
    Mn = orc.Mesh(w.mesh.hex, w.mesh.geom, w.mesh.geom_degree, o_prev, w.flags, orc.params(**w.params), w.mesh.bc_tag)
    _assert_parity(R, Mn.residual(q_prev))


@pytest.mark.parametrize("wall", [3, 4])
def test_walls(wall):
    # no-slip (3) and free-slip (4) walls on a wavy degree-2 channel, mixed flags and orders,
    # every element re-oriented
    w = wl.channel_walls(n=4, wall=wall)
    mesh, _ = wl.rotate_elements(w.mesh, 31 + wall)
    w = small_mixed(dataclasses.replace(w, mesh=mesh), seed=32 + wall, orders=(2, 5))
    p = dict(w.params, nu=1e-2)
    R, R_ref, *_ = _residual_pair(w, params=p)
    _assert_parity(R, R_ref)


def test_padapt_scaled():
    w = wl.padapt_32x32x32(n=6)
    R, R_ref, *_ = _residual_pair(w)
    _assert_parity(R, R_ref)


def test_conservation_and_free_stream_on_gpu():
    w = small_mixed(wl.padapt_32x32x32(n=4), seed=4, orders=(2, 6))
    R, R_ref, M, S, q = _residual_pair(w, params=dict(w.params, nu=1e-2))
    c = S.conservation(to_dev(R))
    scale = np.abs(M.conservation(np.abs(R))).max()
    assert np.abs(c).max() <= 1e-12 * scale
    qc = np.zeros_like(q)
    qc[0], qc[1], qc[2], qc[3] = 0.2, 1.0, 0.3, -0.4
    Rc = S.residual(to_dev(qc)).cpu().numpy()
    assert np.abs(Rc).max() < 1e-11


def test_flags_and_orders_can_change():
    w = small_mixed(wl.tgv_4x4x4_n3(n_elem_dir=4), seed=5)
    M0 = oracle_mesh(w)
    S = gpu_solver(w)
    q = oracle_state(w, M0)
    _assert_parity(S.residual(to_dev(q)).cpu().numpy(), M0.residual(q))
    w2 = small_mixed(w, seed=6, orders=(2, 5))
    S.set_orders(w2.orders)
    S.set_flags(w2.flags)
    M2 = oracle_mesh(w2)
    q2 = oracle_state(w2, M2)
    _assert_parity(S.residual(to_dev(q2)).cpu().numpy(), M2.residual(q2))


def test_mixed_full_size_sampled():
    """64^3 stretched mesh, N = 4, 25% NS, synthetic turbulence: the configuration the
    benchmark times, checked on a sample of elements (the oracle evaluates just those).

    Here R_p = -c0^2 div u of a divergence-free field is ~1 while c0^2 u ~ 25 and the
    smallest cells have 2/h ~ 220, so FP64 itself carries ~3e-12 relative rounding in the
    oracle's weak form; the 1e-12 bar is checked against the extended-precision oracle
    (same source, long double) and the FP64 oracle is checked at its own rounding level."""
    import torch
    w = wl.mixed_64x64x64_n4()
    assert 0.23 < w.ns_fraction < 0.27
    M = oracle_mesh(w)
    xyz = torch.from_numpy(M.node_coords()).cuda()
    # the seeded Fourier field, evaluated with torch on the device for speed (input only)
    q = torch.zeros((4, M.total), dtype=torch.float64, device="cuda")
    q[1:] = _fourier_torch(w, xyz)
    q[1] += 1.0
    del xyz
    S = gpu_solver(w)
    R = S.residual(q).cpu().numpy()
    qh = q.cpu().numpy()
    rng = np.random.default_rng(0)
    ns = np.flatnonzero(w.flags)
    eu = np.flatnonzero(w.flags == 0)
    sel = np.concatenate([rng.choice(ns, 24, replace=False), rng.choice(eu, 24, replace=False), [0, w.n_elem - 1]])
    idx = np.concatenate([np.arange(M.offsets[e], M.offsets[e + 1]) for e in sel])
    R64 = np.zeros_like(qh)
    M.residual(qh, sel=sel, out=R64)
    m = w.mesh
    from oracle import oracle as orc
    Mx = orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, orc.params(**w.params), m.bc_tag, extended=True)
    Rx = np.zeros_like(qh)
    Mx.residual(qh, sel=sel, out=Rx)
    _assert_parity(R[:, idx], Rx[:, idx])
    assert rel_l2(R64[:, idx], Rx[:, idx]) < 1e-11  # the FP64 oracle's own rounding here
    assert rel_l2(R[:, idx], R64[:, idx]) < 1e-11


def _fourier_torch(w, xyz):
    import torch
    modes = wl.kraichnan_modes(w.seed, (8.0, 4.0, 4.0), nmodes=64, kmin=2 * np.pi / 4.0, kmax=np.pi * 64 / 4.0)
    k = torch.from_numpy(modes.k).cuda()
    amp = torch.from_numpy(modes.amp).cuda()
    ph = torch.from_numpy(modes.phase).cuda()
    out = torch.zeros((3, xyz.shape[1]), dtype=torch.float64, device="cuda")
    for m in range(k.shape[0]):
        out += amp[m][:, None] * torch.cos(k[m] @ xyz + ph[m])[None, :]
    return out


def test_bad_inputs_are_rejected():
    from paper_2403_05463_gb300 import dg
    w = wl.tgv_4x4x4_n3()
    S = gpu_solver(w)
    with pytest.raises(dg.DGError) as ei:
        S.set_orders(np.full(w.n_elem, 9, np.int8))
    assert ei.value.status == 1
    with pytest.raises(dg.DGError):
        S.set_flags(np.full(w.n_elem, 3, np.uint8))
    bad = w.mesh.hex.copy()
    bad[0, 1] = bad[0, 0]  # repeated vertex id on a face
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(bad, w.mesh.geom, 1, w.params)
    assert ei.value.status == 2
    nb = wl.wake_16x16x16_n4(n=3)
    with pytest.raises(dg.DGError) as ei:  # inflow/outflow faces without tags
        dg.Solver(nb.mesh.hex, nb.mesh.geom, 1, nb.params, bc_tag=None)
    assert ei.value.status == 2
    flipped = w.mesh.geom.copy()
    flipped[:, :, 0] *= -1.0  # mirrored elements: negative Jacobian
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(w.mesh.hex, flipped, 1, w.params)
    assert ei.value.status == 2
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(w.mesh.hex, w.mesh.geom, 1, dict(w.params, c0sq=-1.0))
    assert ei.value.status == 1
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(w.mesh.hex, w.mesh.geom, 1, dict(w.params, mixed_face=2))
    assert ei.value.status == 1


def test_host_buffer_variants():
    """dg_residual_host / dg_rk_step_host (split transfers; without g the RK register stays on
    the device) give the device results."""
    import torch
    w = small_mixed(wl.padapt_32x32x32(n=4), seed=90, orders=(2, 4))
    M = oracle_mesh(w)
    q = oracle_state(w, M)
    S = gpu_solver(w)
    R = S.residual(to_dev(q)).cpu().numpy()
    Rh = np.zeros_like(q)
    S.residual_host(q, Rh)
    np.testing.assert_array_equal(Rh, R)
    qd, gd = to_dev(q), torch.zeros((4, S.total_nodes), dtype=torch.float64, device="cuda")
    S.rk_step(qd, gd, 1e-4, 2)
    q1 = q.copy()
    g1 = np.zeros_like(q)
    S.rk_step_host(q1, g1, 1e-4, 2)
    np.testing.assert_array_equal(q1, qd.cpu().numpy())
    np.testing.assert_array_equal(g1, gd.cpu().numpy())
    q2 = torch.from_numpy(q.copy()).pin_memory()
    S.rk_step_host(q2, None, 1e-4, 2)
    np.testing.assert_array_equal(q2.numpy(), qd.cpu().numpy())
