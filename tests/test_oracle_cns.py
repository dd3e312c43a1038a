"""Pins of the compressible form of the oracle (App. A): state u = (rho, rho v, rho e), Roe
flux, BR1 on (v, T), heat flux, Vreman/Smagorinsky eddy viscosity mu_t = rho nu_t.

Pinned against what the mathematics fixes: the flux Jacobian against finite differences and
the Euler flux's homogeneity F(u) = A(u) u; the Roe property A(u_roe)(uR - uL) = F(uR) - F(uL)
with the textbook Roe averages, and |A_roe| against numpy's eigen-decomposition of that
matrix; consistency, conservation and supersonic upwinding of the numerical fluxes; free
stream and conservation of the residual on curved, re-oriented, mixed-flag meshes; Euler = NS
without viscosity; invariance under element re-numbering; spectral convergence to the
symbolic (sympy) residual of the compressible Navier-Stokes equations with heat flux; at
adiabatic walls the mirror identities with the doubled periodic channel, mass and energy
conservation and a tangential free stream; at far-field inflow and pressure outflow faces the
free stream and the identity with the periodic box for a state that is the far field near
them."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2403_05463_gb300 import workloads as wl

GAMMA = 1.4


def _state(rng, n=1):
    rho = rng.uniform(0.5, 2.0, n)
    v = rng.normal(scale=0.8, size=(3, n))
    p = rng.uniform(0.5, 3.0, n)
    E = p / (GAMMA - 1) + 0.5 * rho * (v ** 2).sum(0)
    return np.vstack([rho, rho * v, E]).T.squeeze()


def _unit(rng):
    n = rng.normal(size=3)
    return n / np.linalg.norm(n)


def _roe_state(uL, uR):
    """A conservative state with the Roe-averaged velocity and enthalpy (textbook definition)."""
    def vh(u):
        v = u[1:4] / u[0]
        p = (GAMMA - 1) * (u[4] - 0.5 * u[0] * v @ v)
        return v, (u[4] + p) / u[0]
    vL, HL = vh(uL)
    vR, HR = vh(uR)
    sL, sR = np.sqrt(uL[0]), np.sqrt(uR[0])
    v = (sL * vL + sR * vR) / (sL + sR)
    H = (sL * HL + sR * HR) / (sL + sR)
    rho = sL * sR
    E = (rho * H + (GAMMA - 1) * 0.5 * rho * v @ v) / GAMMA
    return np.concatenate([[rho], rho * v, [E]])


@pytest.mark.parametrize("seed", range(4))
def test_jacobian_finite_differences_and_homogeneity(seed):
    rng = np.random.default_rng(seed)
    u, n = _state(rng), _unit(rng)
    A = orc.cns_jacobian(u, n, GAMMA)
    h = 1e-6
    Afd = np.zeros((5, 5))
    for j in range(5):
        e = np.zeros(5)
        e[j] = h * max(1.0, abs(u[j]))
        Afd[:, j] = (orc.cns_flux(u + e, n, GAMMA) - orc.cns_flux(u - e, n, GAMMA)) / (2 * e[j])
    np.testing.assert_allclose(A, Afd, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(A @ u, orc.cns_flux(u, n, GAMMA), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_roe_property_and_eigen_decomposition(seed):
    rng = np.random.default_rng(10 + seed)
    uL, uR, n = _state(rng), _state(rng), _unit(rng)
    A = orc.cns_jacobian(_roe_state(uL, uR), n, GAMMA)
    dF = orc.cns_flux(uR, n, GAMMA) - orc.cns_flux(uL, n, GAMMA)
    np.testing.assert_allclose(A @ (uR - uL), dF, rtol=1e-12, atol=1e-12)
    lam, V = np.linalg.eig(A)
    absA = (V * np.abs(lam)) @ np.linalg.inv(V)
    np.testing.assert_allclose(orc.cns_roe_abs_jacobian(uL, uR, n, GAMMA), absA.real, rtol=1e-10, atol=1e-11)
    # eigenvalues vn -+ a and vn three times at the Roe state
    assert np.allclose(np.sort(lam.real)[1:4], np.sort(lam.real)[2], atol=1e-10)


@pytest.mark.parametrize("riemann", [0, 1])
def test_numerical_flux_consistency_conservation_and_upwinding(riemann):
    rng = np.random.default_rng(20)
    prm = orc.params(riemann=riemann, gamma=GAMMA)
    for _ in range(5):
        u, uR, n = _state(rng), _state(rng), _unit(rng)
        np.testing.assert_allclose(orc.cns_riemann(u, u, n, prm), orc.cns_flux(u, n, GAMMA), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(orc.cns_riemann(u, uR, n, prm), -orc.cns_riemann(uR, u, -n, prm), rtol=1e-12,
                                   atol=1e-12)
    if riemann == 0:
        # supersonic along n on both sides (and at the Roe state): the Roe flux is the left flux
        n = np.array([1.0, 0.0, 0.0])
        def sup(rho, vx, p):
            return np.array([rho, rho * vx, 0.1 * rho, 0.0, p / (GAMMA - 1) + 0.5 * rho * (vx ** 2 + 0.01)])
        uL, uR = sup(1.0, 3.0, 1.0), sup(1.2, 3.2, 1.1)
        np.testing.assert_allclose(orc.cns_riemann(uL, uR, n, prm), orc.cns_flux(uL, n, GAMMA), rtol=1e-13)


def _cns_params(**kw):
    base = dict(nu=0.0, cs=0.1, cv=0.07, closure=1, riemann=0, gamma=GAMMA, prandtl=0.72, prandtl_t=0.9)
    base.update(kw)
    return orc.params(**base)


def _curved_periodic(n=3, order=3, seed=0, rotate=True, flags_p=0.5):
    w = wl.padapt_32x32x32(n=n, amp=0.05)
    rng = np.random.default_rng(seed)
    flags = (rng.uniform(size=n ** 3) < flags_p).astype(np.uint8)
    mesh = w.mesh
    if rotate:
        mesh, _ = wl.rotate_elements(mesh, seed + 7)
    return dataclasses.replace(w, mesh=mesh, orders=np.full(n ** 3, order, np.int8), flags=flags)


def _mesh(w, prm):
    m = w.mesh
    return orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, prm, m.bc_tag)


def test_free_stream_is_preserved_on_curved_reoriented_meshes():
    w = _curved_periodic(order=4, seed=1)
    M = _mesh(w, _cns_params(nu=1e-2))
    u = np.zeros((5, M.total))
    rho, v, p = 1.3, np.array([0.4, -0.2, 0.3]), 2.0
    u[0], u[1:4] = rho, (rho * v)[:, None]
    u[4] = p / (GAMMA - 1) + 0.5 * rho * v @ v
    R = M.cns_residual(u)
    assert np.abs(R).max() < 1e-12


@pytest.mark.parametrize("closure,riemann,mixed_face", [(1, 0, 0), (0, 1, 1)])
def test_conservation_on_periodic_mixed_meshes(closure, riemann, mixed_face):
    w = _curved_periodic(order=3, seed=2)
    M = _mesh(w, _cns_params(nu=5e-3, closure=closure, riemann=riemann, mixed_face=mixed_face))
    u = wl.cns_state(M.node_coords(), seed=3)
    R = M.cns_residual(u)
    s = M.cns_conservation(R)
    J_scale = np.abs(R).max()
    assert np.all(np.abs(s) < 1e-12 * J_scale * 8.0), s  # domain volume 1, |R| scale
    assert np.abs(R).max() > 1e-3  # a non-trivial residual


def test_euler_equals_ns_without_viscosity():
    w = _curved_periodic(order=3, seed=3)
    M0 = _mesh(dataclasses.replace(w, flags=np.zeros_like(w.flags)), _cns_params())
    M1 = _mesh(dataclasses.replace(w, flags=np.ones_like(w.flags)), _cns_params(cs=0.0, closure=0))
    u = wl.cns_state(M0.node_coords(), seed=4)
    R0, R1 = M0.cns_residual(u), M1.cns_residual(u)
    assert np.abs(R1 - R0).max() <= 1e-12 * np.abs(R0).max()
    # and viscosity does matter
    M2 = _mesh(dataclasses.replace(w, flags=np.ones_like(w.flags)), _cns_params(nu=1e-2))
    assert np.abs(M2.cns_residual(u) - R0).max() > 1e-6


def test_invariance_under_element_renumbering():
    w = _curved_periodic(order=3, seed=5, rotate=False)
    prm = _cns_params(nu=1e-2)
    rmesh, rot_of = wl.rotate_elements(w.mesh, 55)
    A = _mesh(w, prm)
    B = _mesh(dataclasses.replace(w, mesh=rmesh), prm)
    xa = A.node_coords()
    perm = np.zeros(A.total, dtype=np.int64)
    for e in range(A.ne):
        n = int(w.orders[e]) + 1
        idx = wl.rotation_index_map(wl.CUBE_ROTATIONS[rot_of[e]], n)
        perm[B.offsets[e]:B.offsets[e + 1]] = A.offsets[e] + idx
    np.testing.assert_allclose(B.node_coords(), xa[:, perm], atol=1e-13)
    u = wl.cns_state(xa, seed=6)
    Ra, Rb = A.cns_residual(u), B.cns_residual(u[:, perm])
    assert np.abs(Rb - Ra[:, perm]).max() <= 1e-12 * np.abs(Ra).max()


def _exact_cns_residual(xyz, mu, prandtl):
    """-div F_e + div F_v of App. A for a smooth periodic state (laminar, constant mu,
    kappa = c_p mu / Pr, T = p / rho), evaluated symbolically (sympy)."""
    import sympy as sp
    x, y, z = sp.symbols("x y z")
    X = [x, y, z]
    rho = 1 + sp.Rational(1, 5) * sp.sin(x) * sp.cos(y) * sp.sin(z)
    v = [sp.sin(x) * sp.cos(y) * sp.cos(z), -sp.cos(x) * sp.sin(y) * sp.cos(z), sp.Rational(3, 10) * sp.sin(z) * sp.cos(x)]
    p = 10 + (sp.cos(2 * x) + sp.cos(2 * y)) * (sp.cos(2 * z) + 2) / 16
    g = sp.Rational(7, 5)
    E = p / (g - 1) + rho * sum(vi ** 2 for vi in v) / 2
    T = p / rho
    cp = g / (g - 1)
    kappa = cp * mu / prandtl
    G = [[sp.diff(v[c], X[k]) for k in range(3)] for c in range(3)]
    div = G[0][0] + G[1][1] + G[2][2]
    tau = [[mu * (G[c][k] + G[k][c]) - (sp.Rational(2, 3) * mu * div if c == k else 0) for k in range(3)]
           for c in range(3)]
    Fe = [[rho * v[k] for k in range(3)]]
    for c in range(3):
        Fe.append([rho * v[c] * v[k] + (p if c == k else 0) for k in range(3)])
    Fe.append([(E + p) * v[k] for k in range(3)])
    Fv = [[0, 0, 0]] + [[tau[c][k] for k in range(3)] for c in range(3)]
    Fv.append([sum(v[j] * tau[j][k] for j in range(3)) + kappa * sp.diff(T, X[k]) for k in range(3)])
    R = [sum(-sp.diff(Fe[i][k], X[k]) + sp.diff(Fv[i][k], X[k]) for k in range(3)) for i in range(5)]
    U = [rho] + [rho * vi for vi in v] + [E]
    fR = sp.lambdify((x, y, z), R, "numpy")
    fU = sp.lambdify((x, y, z), U, "numpy")
    shape = xyz[0].shape
    Rex = np.array([np.broadcast_to(np.asarray(o, dtype=float), shape) for o in fR(*xyz)])
    u = np.array([np.broadcast_to(np.asarray(o, dtype=float), shape) for o in fU(*xyz)])
    return u, Rex


def test_spectral_convergence_to_the_symbolic_residual():
    pytest.importorskip("sympy")
    errs = []
    for N in range(2, 8):
        w = wl.tgv_4x4x4_n3(order=N)
        w = dataclasses.replace(w, flags=np.ones(w.n_elem, np.uint8))
        M = _mesh(w, _cns_params(nu=0.05, cs=0.0, closure=0))
        u, Rex = _exact_cns_residual(M.node_coords(), 0.05, 0.72)
        R = M.cns_residual(u)
        errs.append(np.sqrt(((R - Rex) ** 2).sum() / (Rex ** 2).sum()))
    errs = np.array(errs)
    assert np.all(np.diff(np.log(errs)) < -0.5), errs
    assert errs[-1] < 1e-3, errs


def test_rk_step_conserves_and_keeps_a_uniform_state():
    w = _curved_periodic(order=2, seed=8)
    M = _mesh(w, _cns_params(nu=1e-2))
    u = wl.cns_state(M.node_coords(), seed=9)
    g = np.zeros_like(u)
    J = np.zeros(M.total)
    for e in range(M.ne):
        Je, _ = M.element_geometry(e)
        J[M.element_nodes(e)] = Je
    n = int(w.orders[0]) + 1
    x, wq = orc.lgl(n - 1)
    W = np.einsum('i,j,k->kji', wq, wq, wq).ravel()
    Wall = np.tile(W, M.ne)
    before = (Wall * J * u).sum(axis=1)
    M.cns_rk_step(u, g, 1e-3, 2)
    after = (Wall * J * u).sum(axis=1)
    np.testing.assert_allclose(after, before, rtol=1e-12)


# ---- p-nonconforming faces (mortars, Sec. 3.2) -------------------------------------------------

def _mixed_orders(w, seed, lo=2, hi=5):
    rng = np.random.default_rng(seed)
    return dataclasses.replace(w, orders=rng.integers(lo, hi + 1, size=w.n_elem).astype(np.int8))


def test_mortars_keep_the_free_stream_on_curved_meshes():
    w = _mixed_orders(_curved_periodic(order=3, seed=11), 11)
    assert len(set(w.orders.tolist())) > 2
    M = _mesh(w, _cns_params(nu=1e-2))
    u = np.zeros((5, M.total))
    rho, v, p = 1.3, np.array([0.4, -0.2, 0.3]), 2.0
    u[0], u[1:4] = rho, (rho * v)[:, None]
    u[4] = p / (GAMMA - 1) + 0.5 * rho * v @ v
    assert np.abs(M.cns_residual(u)).max() < 1e-12


@pytest.mark.parametrize("closure,riemann,mixed_face", [(1, 0, 0), (0, 1, 1)])
def test_mortars_conserve(closure, riemann, mixed_face):
    w = _mixed_orders(_curved_periodic(order=3, seed=12), 12)
    M = _mesh(w, _cns_params(nu=5e-3, closure=closure, riemann=riemann, mixed_face=mixed_face))
    u = wl.cns_state(M.node_coords(), seed=13)
    R = M.cns_residual(u)
    assert np.abs(R).max() > 1e-3
    assert np.all(np.abs(M.cns_conservation(R)) < 1e-12 * np.abs(R).max() * 8.0)


def test_mortars_euler_equals_ns_without_viscosity():
    w = _mixed_orders(_curved_periodic(order=3, seed=14), 14)
    M0 = _mesh(dataclasses.replace(w, flags=np.zeros_like(w.flags)), _cns_params())
    M1 = _mesh(dataclasses.replace(w, flags=np.ones_like(w.flags)), _cns_params(cs=0.0, closure=0))
    u = wl.cns_state(M0.node_coords(), seed=15)
    R0 = M0.cns_residual(u)
    assert np.abs(M1.cns_residual(u) - R0).max() <= 1e-12 * np.abs(R0).max()


@pytest.mark.parametrize("nodes", [0, 1], ids=["lobatto", "legendre"])
def test_a_polynomial_state_gives_the_exact_residual_across_mortars(nodes):
    # rho and p constant, v = v0 + A x linear: the state (rho e quadratic) and the fluxes (at
    # most cubic) are exact at N >= 3, every Riemann flux is the physical flux, phi = (v, T) has
    # an exact BR1 gradient (T constant) and tau is constant, so on all-NS elements two layers
    # inside an open box of re-oriented affine elements of orders 3..6
    #   R_rho = -rho tr A, R_m = -rho (A v + v tr A), R_E = -(rho v.A v + Hh tr A) + tau : A,
    # Hh = rho e + p. A wrong interpolation, projection or orientation on a mortar breaks it.
    T = np.array([[1.0, 0.3, -0.1], [0.2, 0.8, 0.25], [-0.15, 0.1, 1.2]])
    b = np.linspace(0.0, 1.0, 7)
    desc = wl.box_mesh(6, 6, 6, b, b, b, periodic=(False, False, False),
                       warp=lambda x, y, z: tuple(T @ np.stack([x, y, z])))
    desc, _ = wl.rotate_elements(desc, 41)
    rng = np.random.default_rng(42)
    orders = rng.integers(3, 7, size=216).astype(np.int8)
    nu = 1e-2
    prm = _cns_params(nu=nu, cs=0.0, closure=0, inflow=(1.0, 0.5, 0.0, 0.0), p_inf=2.0, nodes=nodes)
    M = orc.Mesh(desc.hex, desc.geom, desc.geom_degree, orders, np.ones(216, np.uint8), prm, desc.bc_tag)
    A = 0.3 * rng.normal(size=(3, 3))
    rho, p = 1.2, 2.5
    x = M.node_coords()
    v = np.array([0.5, -0.2, 0.3])[:, None] + A @ x
    u = np.concatenate([np.full((1, M.total), rho), rho * v, (p / (GAMMA - 1) + 0.5 * rho * (v * v).sum(0))[None]])
    R = M.cns_residual(u)
    inner = [i + 6 * (j + 6 * k) for i in (2, 3) for j in (2, 3) for k in (2, 3)]
    assert len({int(orders[e]) for e in inner}) > 1
    idx = np.concatenate([np.arange(M.offsets[e], M.offsets[e + 1]) for e in inner])
    vi, trA = v[:, idx], np.trace(A)
    tau = nu * (A + A.T) - 2.0 / 3.0 * nu * trA * np.eye(3)
    Hh = GAMMA / (GAMMA - 1) * p + 0.5 * rho * (vi * vi).sum(0)
    ex = np.concatenate([np.full((1, idx.size), -rho * trA), -rho * (A @ vi + vi * trA),
                         (-(rho * np.einsum('ip,ij,jp->p', vi, A, vi) + Hh * trA) + (tau * A).sum())[None]])
    # rounding: the cancelling flux-derivative terms are ~1e3 times the residual here (energy
    # fluxes ~10, ||D|| ~ N^2 / h), measured 1e-11 of max |ex| on Gauss points, 8e-12 on Lobatto
    # nodes; a wrong mortar operator or orientation gives O(0.1) errors
    assert np.abs(R[:, idx] - ex).max() <= 5e-11 * np.abs(ex).max()


# ---- adiabatic walls (boundary tags 3 no-slip, 4 free-slip) ----------------------------------

def _cns_mirror_residuals(tag, state, flags_value, nodes=0):
    from test_oracle_pins import _channel
    H = 2.0
    mw, ow = _channel(3, 0.0, H, (tag, tag))      # [0, H] between two walls
    mp, op = _channel(6, -H, 2 * H, None)          # [-H, H], periodic: the mirror extension
    prm = _cns_params(nu=1e-2, nodes=nodes)
    Aw = orc.Mesh(mw.hex, mw.geom, 1, ow, np.full(len(ow), flags_value, np.uint8), prm, mw.bc_tag)
    Ap = orc.Mesh(mp.hex, mp.geom, 1, op, np.full(len(op), flags_value, np.uint8), prm, mp.bc_tag)
    Rw = Aw.cns_residual(state(Aw.node_coords(), H))
    Rp = Ap.cns_residual(state(Ap.node_coords(), H))
    out_w, out_p = [], []
    for e in range(len(ow)):
        i, j, k = e % 3, (e // 3) % 3, e // 9
        ep = i + 3 * ((j + 3) + 6 * k)
        out_w.append(Rw[:, Aw.element_nodes(e)])
        out_p.append(Rp[:, Ap.element_nodes(ep)])
    return np.concatenate(out_w, axis=1), np.concatenate(out_p, axis=1)


def _cns_from_primitive(rho, v, p):
    return np.stack([rho, rho * v[0], rho * v[1], rho * v[2], p / (GAMMA - 1) + 0.5 * rho * (v ** 2).sum(0)])


@pytest.mark.parametrize("flags_value", [0, 1])
def test_free_slip_wall_is_a_mirror(flags_value, nodes=0):
    # rho, p, v_x, v_z even and v_y odd about y = 0 and y = H: the periodic residual of the
    # extended field restricted to [0, H] is the residual between free-slip walls (Euler and NS:
    # the mirror average keeps the normal traction and cancels the normal energy flux)
    def state(x, H):
        c, s = np.cos(np.pi * x[1] / H), np.sin(np.pi * x[1] / H)
        rho = 1.0 + 0.1 * c * np.sin(x[0])
        v = np.stack([0.5 + 0.1 * c * np.sin(x[2]), 0.2 * s * np.cos(x[0]), 0.1 * c * np.cos(x[0])])
        p = 2.0 + 0.2 * c * np.cos(x[2]) + 0.1 * np.cos(2 * np.pi * x[1] / H)
        return _cns_from_primitive(rho, v, p)
    Rw, Rp = _cns_mirror_residuals(4, state, flags_value, nodes)
    assert np.abs(Rw - Rp).max() <= 1e-12 * np.abs(Rp).max()


def test_no_slip_wall_is_an_antimirror_for_euler():
    # rho, p even and every velocity component odd about the walls
    def state(x, H):
        c, s = np.cos(np.pi * x[1] / H), np.sin(np.pi * x[1] / H)
        rho = 1.0 + 0.1 * c * np.cos(x[0])
        v = np.stack([s * (0.5 + 0.1 * np.cos(x[2])), 0.2 * np.sin(2 * np.pi * x[1] / H) * np.cos(x[0]),
                      0.3 * s * np.sin(x[0])])
        p = 2.0 + 0.2 * c * np.sin(x[2])
        return _cns_from_primitive(rho, v, p)
    Rw, Rp = _cns_mirror_residuals(3, state, 0)
    assert np.abs(Rw - Rp).max() <= 1e-12 * np.abs(Rp).max()


@pytest.mark.parametrize("tag", [3, 4])
def test_walls_conserve_mass_and_energy(tag):
    # the mirror ghost makes the Roe mass and energy fluxes through a wall vanish, and the
    # adiabatic wall carries no viscous energy flux: the mass and energy sums stay zero
    from test_oracle_pins import _channel
    mw, ow = _channel(3, 0.0, 2.0, (tag, tag))
    rng = np.random.default_rng(30 + tag)
    flags = rng.integers(0, 2, size=len(ow)).astype(np.uint8)
    M = orc.Mesh(mw.hex, mw.geom, 1, ow, flags, _cns_params(nu=1e-2), mw.bc_tag)
    u = wl.cns_state(M.node_coords(), seed=tag, period=2 * np.pi)
    R = M.cns_residual(u)
    s = M.cns_conservation(R)
    scale = np.abs(R).max()
    assert abs(s[0]) < 1e-12 * scale and abs(s[4]) < 1e-12 * scale, s
    assert np.abs(s[1:4]).max() > 1e-6 * scale  # momentum does cross the walls (pressure, traction)


def test_free_slip_walls_keep_a_tangential_free_stream():
    from test_oracle_pins import _channel
    mw, ow = _channel(3, 0.0, 2.0, (4, 4), N=4)
    M = orc.Mesh(mw.hex, mw.geom, 1, ow, np.ones(len(ow), np.uint8), _cns_params(nu=1e-2), mw.bc_tag)
    xyz = M.node_coords()
    u = _cns_from_primitive(np.full(M.total, 1.2), np.stack([np.full(M.total, 0.6), np.zeros(M.total),
                                                              np.full(M.total, -0.2)]), np.full(M.total, 1.5))
    assert np.abs(M.cns_residual(u)).max() < 1e-12


# ---- far-field inflow (tag 1) and pressure outflow (tag 2) ------------------------------------

FAR = dict(rho=1.1, v=(0.6, 0.1, -0.2), p=1.8)


def _far_params(**kw):
    return _cns_params(inflow=(FAR["rho"], *FAR["v"]), p_inf=FAR["p"], **kw)


def _box_x(periodic_x, n=(5, 3, 3), order=3):
    nx, ny, nz = n
    m = wl.box_mesh(nx, ny, nz, np.linspace(0, 5.0, nx + 1), np.linspace(0, 2 * np.pi, ny + 1),
                    np.linspace(0, 2 * np.pi, nz + 1), periodic=(periodic_x, True, True), bc_lohi=(1, 2))
    return m, np.full(nx * ny * nz, order, np.int8)


@pytest.mark.parametrize("flags_value", [0, 1])
def test_far_field_free_stream_through_inflow_and_outflow(flags_value):
    m, o = _box_x(False)
    M = orc.Mesh(m.hex, m.geom, 1, o, np.full(len(o), flags_value, np.uint8), _far_params(nu=1e-2), m.bc_tag)
    n = M.total
    v = np.stack([np.full(n, c) for c in FAR["v"]])
    u = _cns_from_primitive(np.full(n, FAR["rho"]), v, np.full(n, FAR["p"]))
    assert np.abs(M.cns_residual(u)).max() < 1e-12


def test_inflow_outflow_equal_the_periodic_box_for_euler():
    # the state is the far field in the first and last element layers along x and varies in
    # between: the inflow ghost (far field) and the outflow ghost (interior rho, v and p_inf)
    # then see what the periodic neighbour shows, so every element's residual is the same
    mw, o = _box_x(False)
    mp, _ = _box_x(True)
    prm = _far_params()
    Aw = orc.Mesh(mw.hex, mw.geom, 1, o, np.zeros(len(o), np.uint8), prm, mw.bc_tag)
    Ap = orc.Mesh(mp.hex, mp.geom, 1, o, np.zeros(len(o), np.uint8), prm, mp.bc_tag)
    x = Aw.node_coords()
    np.testing.assert_array_equal(x, Ap.node_coords())
    b = np.where((x[0] > 1.0) & (x[0] < 4.0), np.sin(np.pi * (x[0] - 1.0) / 3.0) ** 2, 0.0)
    rho = FAR["rho"] * (1 + 0.1 * b * np.cos(x[1]))
    v = np.stack([FAR["v"][0] + 0.2 * b * np.sin(x[2]), FAR["v"][1] + 0.1 * b, FAR["v"][2] * (1 + b * np.cos(x[1]))])
    p = FAR["p"] * (1 + 0.05 * b * np.sin(x[1] + x[2]))
    u = _cns_from_primitive(rho, v, p)
    Rw, Rp = Aw.cns_residual(u), Ap.cns_residual(u)
    assert np.abs(Rw - Rp).max() <= 1e-12 * np.abs(Rp).max()
    assert np.abs(Rp).max() > 1e-2


def test_inflow_and_outflow_ghost_states():
    # a uniform interior (rho1, v1, p1) and a different far field: only the face nodes on the
    # inflow and outflow faces feel the ghosts, with R = s/(w_end J) (F(u) - F*(u, u_ghost)) . n;
    # the ghost is the far field at the inflow and (rho1, rho1 v1, p_inf) at the outflow (F* from
    # the pinned Roe flux)
    nx, N = 5, 3
    m, o = _box_x(False, order=N)
    rho1, v1, p1 = 1.1, np.array([0.6, 0.1, -0.2]), 1.8
    rinf, vinf, pinf = 0.9, np.array([0.7, -0.1, 0.05]), 2.1
    prm = _cns_params(inflow=(rinf, *vinf), p_inf=pinf)
    M = orc.Mesh(m.hex, m.geom, 1, o, np.zeros(len(o), np.uint8), prm, m.bc_tag)
    n = M.total
    u1 = _cns_from_primitive(np.array([rho1]), v1[:, None], np.array([p1]))[:, 0]
    R = M.cns_residual(np.repeat(u1[:, None], n, axis=1))
    g_in = _cns_from_primitive(np.array([rinf]), vinf[:, None], np.array([pinf]))[:, 0]
    g_out = _cns_from_primitive(np.array([rho1]), v1[:, None], np.array([pinf]))[:, 0]
    h = 1.0
    w0 = 2.0 / (N * (N + 1))
    for nx_sign, elem_i, node_i, ghost in ((-1.0, 0, 0, g_in), (1.0, nx - 1, N, g_out)):
        nh = np.array([nx_sign, 0.0, 0.0])
        expect = (2.0 / h) / w0 * (orc.cns_flux(u1, nh, GAMMA) - orc.cns_riemann(u1, ghost, nh, prm))
        e = elem_i  # element (elem_i, 0, 0)
        Re = R[:, M.element_nodes(e)].reshape(5, N + 1, N + 1, N + 1)
        np.testing.assert_allclose(Re[:, :, :, node_i], expect[:, None, None] * np.ones((N + 1, N + 1)), rtol=1e-12,
                                   atol=1e-12)
        other = np.delete(Re, node_i, axis=3)
        assert np.abs(other).max() < 1e-12
    # the interior elements see only uniform neighbours
    assert np.abs(R[:, M.element_nodes(2)]).max() < 1e-12


def test_inflow_outflow_need_a_far_field():
    w = wl.wake_16x16x16_n4(n=3, order=2)
    M = _mesh(w, _cns_params())  # no far-field density or pressure given
    with pytest.raises(RuntimeError):
        M.cns_residual(np.ones((5, M.total)))


# ---- Gauss-Legendre nodes (App. B's quadrature) ------------------------------------------------

def test_gauss_legendre_free_stream_conservation_and_euler_limit():
    # curved re-oriented mesh with orders 2..5: free stream, sum w J R = 0 with the Gauss weights
    # (Roe and LLF), and Euler = NS without viscosity
    w = _mixed_orders(_curved_periodic(order=3, seed=16), 16)
    M = _mesh(w, _cns_params(nu=1e-2, nodes=1))
    u = np.zeros((5, M.total))
    rho, v, p = 1.3, np.array([0.4, -0.2, 0.3]), 2.0
    u[0], u[1:4] = rho, (rho * v)[:, None]
    u[4] = p / (GAMMA - 1) + 0.5 * rho * v @ v
    # rounding of terms ~ (rho e + p)|v| ||D|| lifted with l_i(+-1)/w_i: measured 1.6e-12
    assert np.abs(M.cns_residual(u)).max() < 1e-11
    u = wl.cns_state(M.node_coords(), seed=17)
    for riemann in (0, 1):
        Mr = _mesh(w, _cns_params(nu=5e-3, riemann=riemann, nodes=1))
        R = Mr.cns_residual(u)
        assert np.abs(R).max() > 1e-3
        assert np.all(np.abs(Mr.cns_conservation(R)) < 1e-12 * np.abs(R).max() * 8.0)
    M0 = _mesh(dataclasses.replace(w, flags=np.zeros_like(w.flags)), _cns_params(nodes=1))
    M1 = _mesh(dataclasses.replace(w, flags=np.ones_like(w.flags)), _cns_params(cs=0.0, closure=0, nodes=1))
    R0 = M0.cns_residual(u)
    assert np.abs(M1.cns_residual(u) - R0).max() <= 1e-12 * np.abs(R0).max()


def test_gauss_legendre_spectral_convergence_to_the_symbolic_residual():
    pytest.importorskip("sympy")
    errs = []
    for N in range(2, 8):
        w = wl.tgv_4x4x4_n3(order=N)
        w = dataclasses.replace(w, flags=np.ones(w.n_elem, np.uint8))
        M = _mesh(w, _cns_params(nu=0.05, cs=0.0, closure=0, nodes=1))
        u, Rex = _exact_cns_residual(M.node_coords(), 0.05, 0.72)
        R = M.cns_residual(u)
        errs.append(np.sqrt(((R - Rex) ** 2).sum() / (Rex ** 2).sum()))
    errs = np.array(errs)
    assert np.all(np.diff(np.log(errs)) < -0.5), errs
    assert errs[-1] < 1e-3, errs


@pytest.mark.parametrize("flags_value", [0, 1])
def test_gauss_legendre_free_slip_mirror_and_far_field(flags_value):
    test_free_slip_wall_is_a_mirror(flags_value, nodes=1)
    m, o = _box_x(False)
    M = orc.Mesh(m.hex, m.geom, 1, o, np.full(len(o), flags_value, np.uint8), _far_params(nu=1e-2, nodes=1), m.bc_tag)
    n = M.total
    v = np.stack([np.full(n, c) for c in FAR["v"]])
    u = _cns_from_primitive(np.full(n, FAR["rho"]), v, np.full(n, FAR["p"]))
    assert np.abs(M.cns_residual(u)).max() < 1e-12


@pytest.mark.parametrize("nodes", [0, 1], ids=["lobatto", "legendre"])
def test_affine_gradient_of_v_and_T_exact_for_polynomials(nodes):
    # the BR1 gradient of the primitive (v, T) lifts nothing for fields continuous across the
    # element's faces, and the derivative operators are exact for degree <= N on affine maps:
    # on the central element of a sheared 3^3 box it equals the exact gradient (v quadratic in
    # its own coordinate, T linear, rho constant, p = rho T). N = 4, so that on Gauss points the
    # face values interpolated from the conservative state (rho e of degree 4) are exact too
    rng = np.random.default_rng(11)
    n = 3
    b = np.linspace(0, 1, n + 1)
    A = np.array([[1.0, 0.3, 0.0], [0.1, 0.9, 0.2], [0.0, -0.2, 1.1]])
    mesh = wl.box_mesh(n, n, n, b, b, b, warp=lambda x, y, z: tuple(A @ np.stack([x, y, z])))
    E = n ** 3
    M = orc.Mesh(mesh.hex, mesh.geom, 1, np.full(E, 4, np.int8), np.ones(E, np.uint8),
                 _cns_params(nu=1e-3, nodes=nodes))
    xyz = M.node_coords()
    C = rng.normal(size=(3, 3))
    t = rng.normal(size=3) * 0.1
    rho = np.full(M.total, 1.2)
    v = np.stack([0.3 * C[c] @ xyz + 0.1 * xyz[c] ** 2 for c in range(3)])
    T = 1.0 + t @ xyz
    u = _cns_from_primitive(rho, v, rho * T)
    e = 13  # the central element: every neighbour carries the same polynomials
    G = M.cns_element_gradient(u, e)
    x = xyz[:, M.element_nodes(e)]
    for c in range(3):
        for k in range(3):
            ref = 0.3 * C[c, k] + (0.2 * x[c] if c == k else 0.0)
            np.testing.assert_allclose(G[c, k], ref, atol=1e-10)
    for k in range(3):
        np.testing.assert_allclose(G[3, k], t[k], atol=1e-10)
