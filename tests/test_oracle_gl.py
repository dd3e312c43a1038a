"""Pins of the oracle on Gauss-Legendre nodes (the paper's quadrature, App. B): the rule's closed
forms and exactness, the derivative matrix on polynomials, and the residual with interpolated
face values (free stream on curved re-oriented meshes, conservation with the Gauss weights,
Euler = NS without viscosity, invariance under element re-numbering, spectral convergence to
the symbolic Taylor-Green residual), the wall mirror identities, the inflow/outflow free stream,
p-nonconforming faces (Gauss-point interpolation and projection, free stream, conservation and
exactness of linear states across mortars) and what the node set refuses."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2403_05463_gb300 import workloads as wl


def test_gauss_legendre_closed_forms():
    x, w = orc.gl(1)
    np.testing.assert_allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    np.testing.assert_allclose(w, [1.0, 1.0], atol=1e-15)
    x, w = orc.gl(2)
    np.testing.assert_allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("N", range(1, 8))
def test_gauss_legendre_exact_to_degree_2n_plus_1(N):
    x, w = orc.gl(N)
    for k in range(2 * N + 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(w @ x ** k - exact) < 1e-14, (N, k)
    k = 2 * N + 2
    assert abs(w @ x ** k - 2.0 / (k + 1)) > 1e-6
    np.testing.assert_allclose(x, np.polynomial.legendre.leggauss(N + 1)[0], atol=1e-14)


@pytest.mark.parametrize("N", [1, 3, 6])
def test_gauss_legendre_derivative_matrix(N):
    # exact on x^k for k <= N at the Gauss points, rows sum to zero, and it is not the
    # Lobatto matrix (which would differentiate the wrong interpolant)
    x, _ = orc.gl(N)
    D = orc.dmat_gl(N)
    for k in range(N + 1):
        exact = k * x ** (k - 1) if k else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** k, exact, atol=1e-12 * max(1, k * k))
    assert np.abs(D.sum(axis=1)).max() < 1e-13
    assert np.abs(D - orc.dmat(N)).max() > 0.1


def _params(**kw):
    base = dict(nu=0.0, c0sq=25.0, cs=0.1, cv=0.07, closure=0, riemann=0, nodes=1)
    base.update(kw)
    return orc.params(**base)


def _mesh(w, prm):
    m = w.mesh
    return orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, prm, m.bc_tag)


def _curved(order, seed, rotate=True):
    w = wl.padapt_32x32x32(n=3, amp=0.05)
    rng = np.random.default_rng(seed)
    flags = rng.integers(0, 2, size=w.n_elem).astype(np.uint8)
    mesh = w.mesh
    if rotate:
        mesh, _ = wl.rotate_elements(mesh, seed + 100)
    return dataclasses.replace(w, mesh=mesh, orders=np.full(w.n_elem, order, np.int8), flags=flags)


def test_nodes_and_derivative_matrix_on_polynomials():
    # the element's nodes are the Gauss points mapped by the geometry; D is exact to degree N
    w = wl.tgv_4x4x4_n3(n_elem_dir=3, order=4)
    M = _mesh(w, _params())
    x0, _ = orc.gl(4)
    xyz = M.node_coords()[:, M.element_nodes(0)]
    h = 2 * np.pi / 3
    np.testing.assert_allclose(xyz[0, :5], 0.5 * (x0 + 1) * h, atol=1e-13)
    # the metric of the box at the Gauss points: J = (h/2)^3, J dxi_d/dx_d = (h/2)^2
    J, Ja = M.element_geometry(0)
    np.testing.assert_allclose(J, (h / 2) ** 3, rtol=1e-14)
    for d in range(3):
        np.testing.assert_allclose(Ja[d, d], (h / 2) ** 2, rtol=1e-14)
    # a state linear in x has the exact residual of its flux divergence: R_p = -c0^2 du/dx
    q = np.zeros((4, M.total))
    xs = M.node_coords()
    q[1] = 0.1 * np.sin(xs[1]) + 2.0  # u varies only in y: du/dx = 0, uniform in x
    R = M.residual(q)
    assert np.abs(R[0]).max() < 1e-12


def test_free_stream_on_curved_reoriented_meshes():
    for order in (2, 4):
        w = _curved(order, seed=order)
        M = _mesh(w, _params(nu=1e-2, closure=1))
        q = np.zeros((4, M.total))
        q[0], q[1], q[2], q[3] = 0.3, 1.0, -0.5, 0.25
        # rounding of terms of size c0^2 |u| ||D|| / h ~ 1e3 (the Lobatto pin's bound)
        assert np.abs(M.residual(q)).max() < 1e-11, order


@pytest.mark.parametrize("riemann,mixed_face", [(0, 0), (1, 1)])
def test_conservation_with_gauss_weights(riemann, mixed_face):
    w = _curved(3, seed=7)
    M = _mesh(w, _params(nu=1e-2, riemann=riemann, mixed_face=mixed_face))
    q = w.state(M.node_coords())
    R = M.residual(q)
    s = M.conservation(R)
    assert np.abs(R).max() > 1e-2
    assert np.all(np.abs(s) < 1e-12 * np.abs(R).max()), s


def test_euler_equals_ns_without_viscosity():
    w = _curved(3, seed=8)
    M0 = _mesh(dataclasses.replace(w, flags=np.zeros_like(w.flags)), _params())
    M1 = _mesh(dataclasses.replace(w, flags=np.ones_like(w.flags)), _params(cs=0.0))
    q = w.state(M0.node_coords())
    R0, R1 = M0.residual(q), M1.residual(q)
    assert np.abs(R1 - R0).max() <= 1e-12 * np.abs(R0).max()


def test_invariance_under_element_renumbering():
    w = _curved(3, seed=9, rotate=False)
    prm = _params(nu=1e-2)
    rmesh, rot_of = wl.rotate_elements(w.mesh, 91)
    A = _mesh(w, prm)
    B = _mesh(dataclasses.replace(w, mesh=rmesh), prm)
    xa = A.node_coords()
    perm = np.zeros(A.total, dtype=np.int64)
    for e in range(A.ne):
        n = int(w.orders[e]) + 1
        idx = wl.rotation_index_map(wl.CUBE_ROTATIONS[rot_of[e]], n)
        perm[B.offsets[e]:B.offsets[e + 1]] = A.offsets[e] + idx
    np.testing.assert_allclose(B.node_coords(), xa[:, perm], atol=1e-13)
    q = w.state(xa)
    Ra, Rb = A.residual(q), B.residual(q[:, perm])
    assert np.abs(Rb - Ra[:, perm]).max() <= 1e-12 * np.abs(Ra).max()


def test_spectral_convergence_to_the_symbolic_residual():
    pytest.importorskip("sympy")
    from test_oracle_pins import _tgv_exact_residual
    errs = []
    for N in range(2, 8):
        w = wl.tgv_4x4x4_n3(order=N)
        M = _mesh(w, _params(nu=0.01, cs=0.0))
        xyz = M.node_coords()
        R = M.residual(w.state(xyz))
        Rex = _tgv_exact_residual(xyz, 0.01, 25.0)
        errs.append(np.sqrt(((R - Rex) ** 2).sum() / (Rex ** 2).sum()))
    errs = np.array(errs)
    assert np.all(np.diff(np.log(errs)) < -0.5), errs
    assert errs[-1] < 5e-4, errs


def test_what_gauss_legendre_refuses():
    w = _curved(3, seed=10)
    with pytest.raises(ValueError):
        _mesh(w, _params(split=1))


# ---- p-nonconforming faces (mortars, Sec. 3.2) between Gauss point sets ----------------------

@pytest.mark.parametrize("Nl,Nh", [(1, 2), (2, 5), (3, 7)])
def test_gauss_interpolation_and_projection(Nl, Nh):
    # interpolation is exact on degree <= Nl; projecting an interpolant gives it back; the
    # projection is the truncated Legendre series of the high-degree polynomial (numpy)
    xl, _ = orc.gl(Nl)
    xh, _ = orc.gl(Nh)
    I, P = orc.interp_gl(Nl, Nh), orc.project_gl(Nh, Nl)
    for k in range(Nl + 1):
        np.testing.assert_allclose(I @ xl ** k, xh ** k, atol=1e-13)
    np.testing.assert_allclose(P @ I, np.eye(Nl + 1), atol=1e-13)
    rng = np.random.default_rng(Nh)
    f = rng.normal(size=Nh + 1)
    c = np.polynomial.legendre.legfit(xh, f, Nh)
    np.testing.assert_allclose(P @ f, np.polynomial.legendre.legval(xl, c[:Nl + 1]), atol=1e-12)


def _mixed_orders(w, seed, lo=2, hi=5):
    rng = np.random.default_rng(seed)
    return dataclasses.replace(w, orders=rng.integers(lo, hi + 1, size=w.n_elem).astype(np.int8))


def test_free_stream_on_a_curved_mixed_order_mesh():
    w = _mixed_orders(_curved(3, seed=21), 21)
    M = _mesh(w, _params(nu=1e-2, closure=1))
    q = np.zeros((4, M.total))
    q[0], q[1], q[2], q[3] = 0.3, 1.0, -0.5, 0.25
    assert np.abs(M.residual(q)).max() < 1e-11


@pytest.mark.parametrize("riemann,mixed_face", [(0, 0), (1, 1)])
def test_conservation_on_mixed_orders(riemann, mixed_face):
    w = _mixed_orders(_curved(3, seed=22), 22)
    M = _mesh(w, _params(nu=1e-2, riemann=riemann, mixed_face=mixed_face))
    q = w.state(M.node_coords())
    R = M.residual(q)
    assert np.abs(R).max() > 1e-2
    assert np.all(np.abs(M.conservation(R)) < 1e-12 * np.abs(R).max())


def test_euler_equals_ns_without_viscosity_on_mixed_orders():
    w = _mixed_orders(_curved(3, seed=23), 23)
    M0 = _mesh(dataclasses.replace(w, flags=np.zeros_like(w.flags)), _params())
    M1 = _mesh(dataclasses.replace(w, flags=np.ones_like(w.flags)), _params(cs=0.0))
    q = w.state(M0.node_coords())
    assert np.abs(M1.residual(q) - M0.residual(q)).max() <= 1e-12 * np.abs(M0.residual(q)).max()


@pytest.mark.parametrize("nodes", [0, 1], ids=["lobatto", "legendre"])
def test_a_linear_state_gives_the_exact_residual_across_mortars(nodes):
    # q = (p0 + g.x, u0 + A x) is continuous, so every Riemann flux is the physical flux, the
    # flux u u^T + p I is quadratic (exact at N >= 2) and tau is constant (all elements NS, no
    # eddy viscosity), so BR1 averages it exactly: on elements two layers
    # from the boundary R = -div F exactly, R_p = -c0^2 tr A, R_u = -(A u + u tr A) - g, through
    # faces between orders 2..5 of re-oriented affine elements. A wrong interpolation,
    # projection or orientation on a mortar breaks it.
    T = np.array([[1.0, 0.3, -0.1], [0.2, 0.8, 0.25], [-0.15, 0.1, 1.2]])
    b = np.linspace(0.0, 1.0, 7)
    desc = wl.box_mesh(6, 6, 6, b, b, b, periodic=(False, False, False),
                       warp=lambda x, y, z: tuple(T @ np.stack([x, y, z])))
    desc, _ = wl.rotate_elements(desc, 31)
    rng = np.random.default_rng(32)
    orders = rng.integers(2, 6, size=216).astype(np.int8)
    flags = np.ones(216, np.uint8)  # all NS: an Euler-NS face halves the viscous flux by design
    c0sq = 25.0
    M = orc.Mesh(desc.hex, desc.geom, desc.geom_degree, orders, flags,
                 _params(nu=1e-2, cs=0.0, nodes=nodes, c0sq=c0sq), desc.bc_tag)
    A = rng.normal(size=(3, 3))
    g = rng.normal(size=3)
    x = M.node_coords()
    u = np.array([1.0, -0.5, 0.3])[:, None] + A @ x
    q = np.concatenate([(0.2 + g @ x)[None], u])
    R = M.residual(q)
    inner = [i + 6 * (j + 6 * k) for i in (2, 3) for j in (2, 3) for k in (2, 3)]
    assert len({int(orders[e]) for e in inner}) > 1
    idx = np.concatenate([np.arange(M.offsets[e], M.offsets[e + 1]) for e in inner])
    ex_p = -c0sq * np.trace(A) * np.ones(idx.size)
    ex_u = -(A @ u[:, idx] + u[:, idx] * np.trace(A)) - g[:, None]
    scale = np.abs(ex_u).max()
    assert np.abs(R[0, idx] - ex_p).max() <= 1e-11 * abs(ex_p[0])
    assert np.abs(R[1:, idx] - ex_u).max() <= 1e-11 * scale


@pytest.mark.parametrize("flags_value", [0, 1])
def test_free_slip_wall_is_a_mirror(flags_value):
    # the Lobatto pin on Gauss points: interpolation to the wall commutes with the reflection
    from test_oracle_pins import _mirror_residuals
    def state(x, H):
        c, s = np.cos(np.pi * x[1] / H), np.sin(np.pi * x[1] / H)
        return np.stack([c * (0.3 + 0.1 * np.sin(x[0])), 1.0 + 0.2 * c * np.sin(x[2]), 0.3 * s * np.cos(x[0]),
                         0.2 * c * np.cos(x[0]) + 0.1 * np.cos(2 * np.pi * x[1] / H)])
    Rw, Rp = _mirror_residuals(4, state, flags_value, nodes=1)
    assert np.abs(Rw - Rp).max() <= 1e-12 * np.abs(Rp).max()


def test_no_slip_wall_is_an_antimirror_for_euler():
    from test_oracle_pins import _mirror_residuals
    def state(x, H):
        c, s = np.cos(np.pi * x[1] / H), np.sin(np.pi * x[1] / H)
        return np.stack([c * (0.2 + 0.1 * np.cos(x[0])), s * (1.0 + 0.1 * np.cos(x[2])),
                         0.2 * np.sin(2 * np.pi * x[1] / H) * np.cos(x[0]), 0.3 * s * np.sin(x[0])])
    Rw, Rp = _mirror_residuals(3, state, 0, nodes=1)
    assert np.abs(Rw - Rp).max() <= 1e-12 * np.abs(Rp).max()


def test_inflow_outflow_free_stream():
    w = wl.wake_16x16x16_n4(n=3, order=3)
    M = _mesh(w, _params())
    q = np.zeros((4, M.total))
    q[1] = 1.0
    assert np.abs(M.residual(q)).max() < 1e-12
