"""Pins of the oracle's inflow (boundary tag 1) and outflow (tag 2) faces of the incompressible
form, on Gauss-Lobatto and on Gauss-Legendre nodes (no GPU needed).

Sec. 2.3 couples an element to whatever lies behind a face through the numerical fluxes only, so
a boundary face is a ghost state fed to the same Roe flux and BR1 average. The readings pinned
here: the inflow ghost is the prescribed velocity with the interior pressure, the outflow ghost
the interior velocity with zero pressure, and both faces take the interior viscous flux. Three
independent pins:

* a uniform interior state that differs from both ghosts: only the boundary face nodes feel the
  ghosts, with the face term s / (J w_end) (F_n(q) - F*(q, q_ghost)) on Lobatto nodes (lifted
  with l_i(-+1) / w_i on Gauss nodes), F* written out here from the artificial-compressibility
  Jacobian and numpy's eigen-decomposition, not from the oracle;
* a state that equals the inflow ghost next to both ends: the residual equals that of the same
  box made periodic in x, element by element (Euler and Navier-Stokes elements);
* a divergence-free linear shear whose velocity is the inflow velocity on the inflow face: the
  BR1 gradient is then exact and the stress constant, so the viscous part of the residual
  (Navier-Stokes minus Euler flags) vanishes everywhere only if both faces take the interior
  viscous flux.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2403_05463_gb300 import workloads as wl

C0SQ = 25.0
INFLOW_U = np.array([1.2, -0.05, 0.1])


def _box(nx, order, periodic_x=False):
    m = wl.box_mesh(nx, 3, 3, np.linspace(0.0, float(nx), nx + 1), np.linspace(0.0, 3.0, 4),
                    np.linspace(0.0, 3.0, 4), periodic=(periodic_x, True, True), bc_lohi=(1, 2))
    return m, np.full(nx * 9, order, np.int8)


def _prm(nodes, **kw):
    base = dict(nu=0.0, c0sq=C0SQ, cs=0.1, inflow=(0.0, *INFLOW_U), nodes=nodes)
    base.update(kw)
    return orc.params(**base)


def _oracle(m, o, flags_value, prm):
    return orc.Mesh(m.hex, m.geom, 1, o, np.full(len(o), flags_value, np.uint8), prm, m.bc_tag)


def _flux(q, n):
    # artificial-compressibility normal flux: (c0^2 u.n, u (u.n) + p n)
    un = q[1:] @ n
    return np.concatenate([[C0SQ * un], q[1:] * un + q[0] * n])


def _jacobian(q, n):
    u, un = q[1:], q[1:] @ n
    A = np.zeros((4, 4))
    A[0, 1:] = C0SQ * n
    A[1:, 0] = n
    A[1:, 1:] = un * np.eye(3) + np.outer(u, n)
    return A


def _roe(qm, qp, n):
    # 1/2 (F(q-) + F(q+)) - 1/2 |A(mean)| (q+ - q-), |A| = V |Lambda| V^-1 by numpy
    lam, V = np.linalg.eig(_jacobian(0.5 * (qm + qp), n))
    absA = (V * np.abs(lam)) @ np.linalg.inv(V)
    return 0.5 * (_flux(qm, n) + _flux(qp, n)) - 0.5 * np.real(absA) @ (qp - qm)


def _face_lift(nodes, N):
    """l_i(-1) / w_i, the weight with which a face term at xi = -1 reaches node i (Lobatto: 1/w_0
    at the end node and 0 elsewhere)."""
    x, w = (orc.lgl if nodes == 0 else orc.gl)(N)
    l = np.array([np.prod([(-1.0 - x[j]) / (x[i] - x[j]) for j in range(N + 1) if j != i]) for i in range(N + 1)])
    return l / w


@pytest.mark.parametrize("nodes", [0, 1])
def test_uniform_state_feels_both_ghosts(nodes):
    nx, N, h = 4, 3, 1.0
    m, o = _box(nx, N)
    M = _oracle(m, o, 0, _prm(nodes))
    q1 = np.array([0.7, 0.8, 0.15, -0.1])
    R = M.residual(np.repeat(q1[:, None], M.total, axis=1))
    g_in = np.concatenate([[q1[0]], INFLOW_U])    # prescribed velocity, interior pressure
    g_out = np.concatenate([[0.0], q1[1:]])       # interior velocity, zero pressure
    lift = _face_lift(nodes, N)
    for sign, ex, ghost, lw in ((-1.0, 0, g_in, lift), (1.0, nx - 1, g_out, lift[::-1])):
        n = np.array([sign, 0.0, 0.0])
        face = (2.0 / h) * (_flux(q1, n) - _roe(q1, ghost, n))
        assert np.abs(face).max() > 0.1  # the ghost differs from the interior state
        for ey in range(3):
            for ez in range(3):
                e = ex + nx * (ey + 3 * ez)
                Re = R[:, M.element_nodes(e)].reshape(4, N + 1, N + 1, N + 1)  # [v][k][j][i]
                expect = face[:, None, None, None] * lw[None, None, None, :] * np.ones((4, N + 1, N + 1, N + 1))
                np.testing.assert_allclose(Re, expect, rtol=1e-12, atol=1e-12)
    # elements away from the two ends see uniform neighbours only
    for ex in range(1, nx - 1):
        assert np.abs(R[:, M.element_nodes(ex)]).max() < 1e-12


@pytest.mark.parametrize("nodes", [0, 1])
@pytest.mark.parametrize("flags_value", [0, 1])
def test_inflow_ghost_next_to_both_ends_equals_the_periodic_box(nodes, flags_value):
    # q = (0, inflow velocity) for x < 2 and x > 4, a smooth bump in between: the inflow ghost
    # (interior p = 0, prescribed velocity) and the outflow ghost (interior velocity, p = 0) then
    # are exactly what the periodic neighbour shows, the first two element layers have zero
    # gradient (so the interior viscous flux is the periodic average), and every element's
    # residual is that of the periodic box
    nx, N = 6, 3
    mw, o = _box(nx, N)
    mp, _ = _box(nx, N, periodic_x=True)
    prm = _prm(nodes, nu=1e-2)
    Aw, Ap = _oracle(mw, o, flags_value, prm), _oracle(mp, o, flags_value, prm)
    x = Aw.node_coords()
    np.testing.assert_array_equal(x, Ap.node_coords())
    b = np.where((x[0] > 2.0) & (x[0] < 4.0), np.sin(np.pi * (x[0] - 2.0) / 2.0) ** 2, 0.0)
    q = np.stack([0.3 * b * np.cos(x[1]), INFLOW_U[0] + 0.2 * b * np.sin(x[2]), INFLOW_U[1] + 0.1 * b * np.cos(x[1]),
                  INFLOW_U[2] * (1.0 + b * np.sin(x[1] + x[2]))])
    Rw, Rp = Aw.residual(q), Ap.residual(q)
    assert np.abs(Rp).max() > 1e-2
    assert np.abs(Rw - Rp).max() <= 1e-12 * np.abs(Rp).max()


@pytest.mark.parametrize("nodes", [0, 1])
def test_linear_shear_takes_the_interior_viscous_flux(nodes):
    # u = inflow + x (0, 0.4, -0.3): divergence-free, equal to the inflow velocity at x = 0, so
    # u* is the interior value on every face (the inflow ghost's velocity is the interior one
    # there, the outflow ghost takes the interior velocity) and the BR1 gradient is exact; the
    # stress is constant, its divergence and every interior face term cancel, and the viscous
    # part vanishes only if F_v* is the interior viscous flux at both boundary faces
    nx, N = 4, 3
    m, o = _box(nx, N)
    prm = _prm(nodes, nu=1e-2, cs=0.1)
    ns, eu = _oracle(m, o, 1, prm), _oracle(m, o, 0, prm)
    x = ns.node_coords()
    q = np.stack([0.3 + 0.1 * x[1], INFLOW_U[0] + 0.0 * x[0], INFLOW_U[1] + 0.4 * x[0], INFLOW_U[2] - 0.3 * x[0]])
    G = ns.element_gradient(q, 0)
    np.testing.assert_allclose(G.reshape(3, 3, -1)[1, 0], 0.4, atol=1e-12)
    np.testing.assert_allclose(G.reshape(3, 3, -1)[2, 0], -0.3, atol=1e-12)
    Rns, Reu = ns.residual(q), eu.residual(q)
    assert np.abs(Reu).max() > 1e-2
    # the size of one face term the readings cancel: tau_xy s / (J w) with nu alone
    scale = 1e-2 * 0.4 * 2.0 * np.abs(_face_lift(nodes, N)).max()
    assert np.abs(Rns - Reu).max() <= 1e-10 * scale, np.abs(Rns - Reu).max() / scale
