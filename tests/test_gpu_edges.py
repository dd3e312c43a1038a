"""Edge cases of the hot path on the GPU, through the C ABI, against the oracle: one element
with boundary faces on every side at every order (FP64 and the FP32 path), all-Euler flags
(no viscous launch) and a single NS element among Euler ones (a viscous bucket of one), the
largest order jump across one face (1 against 7), zero RK steps, and an empty mesh (rejected).
FP64 results must meet the 1e-12 relative L2 bar; the FP32 path reports its error against a
regression bound."""
import numpy as np
import pytest

from helpers import rel_l2, to_dev
from oracle import oracle as orc
from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12
PARAMS = dict(nu=1e-2, c0sq=25.0, cs=0.1, cv=0.07, closure=0, riemann=0, inflow=(0.0, 1.0, 0.0, 0.0))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _state(x):
    # a smooth non-polynomial field, so every order sees a different residual
    return np.stack([0.2 * np.cos(x[0] + 0.5 * x[1]), 1.0 + 0.3 * np.sin(x[1]) * np.cos(x[2]),
                     0.2 * np.sin(x[0] * 1.3 + x[2]), 0.1 * np.cos(2.0 * x[1] - x[0])])


def _open_box(nx, lengths=(1.0, 0.8, 1.2), tags=(3, 4)):
    # low faces no-slip walls, high faces free-slip walls in every direction
    xb = np.linspace(0.0, lengths[0], nx + 1)
    yb = np.linspace(0.0, lengths[1], 2)
    zb = np.linspace(0.0, lengths[2], 2)
    return wl.box_mesh(nx, 1, 1, xb, yb, zb, periodic=(False, False, False), bc_lohi=tags)


def _pair(desc, orders, flags, params, precision):
    from paper_2403_05463_gb300 import dg
    M = orc.Mesh(desc.hex, desc.geom, desc.geom_degree, orders, flags, orc.params(**params), desc.bc_tag)
    S = dg.Solver(desc.hex, desc.geom, desc.geom_degree, params, orders, flags, desc.bc_tag, precision=precision)
    return M, S


@pytest.mark.parametrize("N", range(1, 8))
def test_one_element_with_walls_on_every_face(N):
    desc = _open_box(1)
    orders, flags = np.array([N], np.int8), np.array([1], np.uint8)
    M, S = _pair(desc, orders, flags, PARAMS, 0)
    q = _state(M.node_coords())
    R_ref = M.residual(q)
    assert rel_l2(S.residual(to_dev(q)).cpu().numpy(), R_ref) <= TOL
    _, S32 = _pair(desc, orders, flags, PARAMS, 1)
    err = rel_l2(S32.residual(to_dev(q)).cpu().numpy(), R_ref)
    print(f"one element N={N}: FP32 relative L2 error {err:.2e}")
    assert err <= 1e-6, err  # measured 6e-8 .. 9e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_all_euler_and_a_single_ns_element(precision):
    w = wl.tgv_4x4x4_n3(n_elem_dir=5, order=3)
    m = w.mesh
    for flags in (np.zeros(w.n_elem, np.uint8), np.eye(1, w.n_elem, 62, dtype=np.uint8).ravel()):
        M, S = _pair(m, w.orders, flags, dict(w.params, nu=1e-2), precision)
        q = w.state(M.node_coords())
        R_ref = M.residual(q)
        err = rel_l2(S.residual(to_dev(q)).cpu().numpy(), R_ref)
        assert err <= (TOL if precision == 0 else 5e-5), (int(flags.sum()), err)
        g = np.zeros_like(q)
        qd, gd = to_dev(q), to_dev(g)
        S.rk_step(qd, gd, 1e-3, 2)
        M.rk_step(q, g, 1e-3, 2)
        q0 = w.state(M.node_coords())
        err = rel_l2(qd.cpu().numpy() - q0, q - q0)
        assert err <= (1e-11 if precision == 0 else 5e-5), (int(flags.sum()), err)


def test_largest_order_jump_on_one_face():
    desc = _open_box(2, lengths=(2.0, 0.8, 1.2))
    for orders in (np.array([1, 7], np.int8), np.array([7, 1], np.int8)):
        for flags in (np.array([1, 1], np.uint8), np.array([1, 0], np.uint8)):
            M, S = _pair(desc, orders, flags, PARAMS, 0)
            q = _state(M.node_coords())
            assert rel_l2(S.residual(to_dev(q)).cpu().numpy(), M.residual(q)) <= TOL, (orders, flags)


def test_zero_steps_leave_the_state_alone():
    import torch
    w = wl.tgv_4x4x4_n3()
    M, S = _pair(w.mesh, w.orders, w.flags, w.params, 0)
    q = w.state(M.node_coords())
    qd, gd = to_dev(q), torch.zeros((4, S.total_nodes), dtype=torch.float64, device="cuda")
    S.rk_step(qd, gd, 1e-3, 0)
    torch.cuda.synchronize()
    assert np.array_equal(qd.cpu().numpy(), q)


def test_an_empty_mesh_is_rejected():
    from paper_2403_05463_gb300 import dg
    with pytest.raises(dg.DGError) as ei:
        dg.Solver(np.zeros((0, 8), np.int64), np.zeros((0, 8, 3)), 1, PARAMS)
    assert dg.STATUS[ei.value.status] == "DG_ERR_ARG"


def _forced(tmp_path, N, stage_choice, vsplit=0):
    # default tile shapes; the stage form forced (0 separate launches, 2 one launch with tile queues)
    import torch
    path = tmp_path / f"stage_{N}_{stage_choice}_{vsplit}.txt"
    dev = torch.cuda.get_device_name(0)
    with open(path, "w") as f:
        for ps, choice in ((0, "0\t0\t0"), (1, "0\t0\t0"), (2, f"{stage_choice}\t{vsplit}\t0")):
            f.write(f"{dev}\t{ps}\t{N}\t0\t{choice}\n")
    return str(path)


@pytest.mark.parametrize("N", [1, 4, 7])
@pytest.mark.parametrize("nx,flag", [(1, 1), (1, 0), (2, 1)])
def test_tile_queue_stage_kernel_on_tiny_meshes(N, nx, flag, tmp_path):
    # one or two elements with walls: a few tiles against hundreds of persistent blocks, so most
    # blocks claim no tile at all (an empty tile -1 ends their queue) and the inviscid tiles wait
    # on one or two viscous ones; chained steps must match the separate launches bitwise
    import torch
    desc = _open_box(nx)
    orders, flags = np.full(nx, N, np.int8), np.full(nx, flag, np.uint8)
    out = []
    for choice, vsplit in ((0, 0), (2, 0), (2, 3)):
        M, S = _pair(desc, orders, flags, PARAMS, 1)
        rep = S.autotune(_forced(tmp_path, N, choice, vsplit))
        assert ("tile queues" in rep) == (choice == 2), rep
        q = _state(M.node_coords())
        qd, gd = to_dev(q), torch.zeros((4, q.shape[1]), dtype=torch.float64, device="cuda")
        S.rk_step(qd, gd, 1e-4, 3)
        S.check_device()
        out.append(qd)
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[2])
