"""Pins of the region-detection oracle (Sec. 2.1) against what the mathematics fixes: exact
gradients of linear and quadratic fields on box, affine and curved elements; the invariants'
closed forms through eigenvalues, the curl and frame invariance; the mixture posterior against
scipy's and scikit-learn's independent implementations and its special cases; the element
means by brute force on a tiny element; a wake whose shear layer must be found."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from oracle import regions as rg
from paper_2403_05463_gb300 import workloads as wl


def _gmm(w=(0.5, 0.5), means=((0, 0, 0), (-0.1, 0, 0.1)), covs=None, viscous=1):
    if covs is None:
        covs = (np.diag([1e-4, 1e-6, 1e-4]), np.diag([1e-2, 1e-4, 1e-2]))
    return {"weights": np.array(w, float), "means": np.array(means, float), "covs": np.array(covs, float),
            "viscous": viscous}


def _mesh(desc, orders, flags=None, nodes=0):
    E = desc.hex.shape[0]
    orders = np.broadcast_to(np.asarray(orders, np.int8), (E,)).copy()
    flags = np.zeros(E, np.uint8) if flags is None else flags
    return orc.Mesh(desc.hex, desc.geom, desc.geom_degree, orders, flags, orc.params(nodes=nodes), desc.bc_tag)


def _open_box(n=3, warp=None, geom_degree=1):
    b = np.linspace(0.0, 1.0, n + 1)
    return wl.box_mesh(n, n, n, b, b, b, periodic=(False, False, False), geom_degree=geom_degree, warp=warp)


def _linear_state(M, A, b0):
    xyz = M.node_coords()
    q = np.zeros((4, M.total))
    q[1:4] = A @ xyz + np.asarray(b0)[:, None]
    return q


def _affine_warp():
    T = np.array([[1.0, 0.3, -0.1], [0.2, 0.8, 0.25], [-0.15, 0.1, 1.2]])
    return lambda x, y, z: tuple(T @ np.stack([x, y, z]))


def _trilinear_warp():
    # multilinear in (x, y, z): the products X_l dX_m/dxi of the curl-form metric terms stay
    # within degree 2 per direction, so the degree-2 geometry gives exact, node-varying metrics
    return lambda x, y, z: (x + 0.3 * y * z, y + 0.2 * x * z, z + 0.25 * x * y)


@pytest.mark.parametrize("nodes", [0, 1], ids=["lobatto", "legendre"])
@pytest.mark.parametrize("kind,orders", [("box", 1), ("box", 3), ("affine", 2), ("rotated", 3),
                                         ("trilinear", 2), ("trilinear", 4)])
def test_gradient_of_a_linear_field_is_exact(kind, orders, nodes):
    # u = A x + b is multilinear in xi on these maps and the metric terms are exact, so the
    # chain rule returns A at every node (per-node metrics on the trilinear map), on either
    # node set (the paper's detection runs on Gauss-Legendre points)
    warp = {"box": None, "affine": _affine_warp(), "rotated": _affine_warp(), "trilinear": _trilinear_warp()}[kind]
    desc = _open_box(3, warp, geom_degree=2 if kind == "trilinear" else 1)
    if kind == "rotated":
        desc, _ = wl.rotate_elements(desc, 5)
    M = _mesh(desc, orders, nodes=nodes)
    rng = np.random.default_rng(11)
    A = rng.normal(size=(3, 3))  # not symmetric: a transposed gradient fails
    q = _linear_state(M, A, rng.normal(size=3))
    for e in range(M.ne):
        G = rg.element_velocity_gradient(M, q, e)
        assert np.abs(G - A[:, :, None]).max() <= 1e-12 * np.abs(A).max(), (kind, e)


@pytest.mark.parametrize("nodes", [0, 1], ids=["lobatto", "legendre"])
def test_gradient_of_a_quadratic_field_on_an_affine_element(nodes):
    # u_c = x . H_c x has d u_c / d x_k = ((H_c + H_c^T) x)_k; degree 2 is exact at N = 2
    desc = _open_box(2, _affine_warp())
    M = _mesh(desc, 2, nodes=nodes)
    rng = np.random.default_rng(12)
    H = rng.normal(size=(3, 3, 3))
    xyz = M.node_coords()
    q = np.zeros((4, M.total))
    for c in range(3):
        q[1 + c] = np.einsum('ip,ij,jp->p', xyz, H[c], xyz)
    for e in range(M.ne):
        x = xyz[:, M.element_nodes(e)]
        exact = np.stack([(H[c] + H[c].T) @ x for c in range(3)])
        G = rg.element_velocity_gradient(M, q, e)
        assert np.abs(G - exact).max() <= 1e-11


def test_invariants_of_a_symmetric_gradient_from_its_eigenvalues():
    rng = np.random.default_rng(13)
    B = rng.normal(size=(50, 3, 3))
    S = 0.5 * (B + np.swapaxes(B, 1, 2))
    lam = np.linalg.eigvalsh(S)
    F = rg.invariants(np.moveaxis(S, 0, -1))
    l1, l2, l3 = lam.T
    np.testing.assert_allclose(F[0], l1 * l2 + l2 * l3 + l3 * l1, atol=1e-12)
    np.testing.assert_allclose(F[1], -l1 * l2 * l3 / 3.0, atol=1e-12)
    assert np.abs(F[2]).max() <= 1e-15  # no rotation


def test_rotation_invariant_is_a_quarter_of_the_squared_vorticity():
    rng = np.random.default_rng(14)
    G = rng.normal(size=(3, 3, 40))
    curl = np.stack([G[2, 1] - G[1, 2], G[0, 2] - G[2, 0], G[1, 0] - G[0, 1]])
    F = rg.invariants(G)
    np.testing.assert_allclose(F[2], (curl ** 2).sum(axis=0) / 4.0, rtol=1e-13)
    # a solid-body rotation u = w x r: no strain, Q_Omega = |w|^2
    w = np.array([0.3, -1.2, 0.7])
    Wx = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    F = rg.invariants(Wx[:, :, None])
    assert abs(F[0, 0]) < 1e-15 and abs(F[1, 0]) < 1e-15
    assert abs(F[2, 0] - w @ w) < 1e-14


def test_pure_strain_closed_form():
    a, b, c = 0.7, -0.2, -0.5
    F = rg.invariants(np.diag([a, b, c])[:, :, None])[:, 0]
    assert abs(F[0] - (a * b + b * c + c * a)) < 1e-15
    assert abs(F[1] + a * b * c / 3.0) < 1e-15
    assert F[2] == 0.0


def test_invariants_do_not_depend_on_the_frame():
    rng = np.random.default_rng(15)
    G = rng.normal(size=(3, 3))
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    F0 = rg.invariants(G[:, :, None])[:, 0]
    F1 = rg.invariants((Q @ G @ Q.T)[:, :, None])[:, 0]
    np.testing.assert_allclose(F1, F0, atol=1e-13)
    # and for an incompressible gradient they add up to the Q-criterion -tr(G^2)/2
    G0 = G - np.trace(G) / 3.0 * np.eye(3)
    F = rg.invariants(G0[:, :, None])[:, 0]
    assert abs(F[0] + F[2] + 0.5 * np.trace(G0 @ G0)) < 1e-13


def _random_gmm(rng, viscous=1):
    covs = []
    for _ in range(2):
        B = rng.normal(size=(3, 3))
        covs.append(B @ B.T + 0.3 * np.eye(3))
    return _gmm(w=rng.uniform(0.2, 0.8, 2), means=rng.normal(size=(2, 3)), covs=covs, viscous=viscous)


def test_gaussian_log_density_against_scipy():
    st = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(16)
    g = _random_gmm(rng)
    X = rng.normal(scale=2.0, size=(3, 30))
    for k in range(2):
        ref = st.multivariate_normal(mean=g["means"][k], cov=g["covs"][k]).logpdf(X.T)
        np.testing.assert_allclose(rg.gaussian_log_density(X, g["means"][k], g["covs"][k]), ref, rtol=1e-13)


def test_memberships_against_scikit_learn():
    mix = pytest.importorskip("sklearn.mixture")
    rng = np.random.default_rng(17)
    g = _random_gmm(rng, viscous=0)
    X = rng.normal(scale=1.5, size=(3, 60))
    gm = mix.GaussianMixture(n_components=2, covariance_type="full")
    gm.weights_ = g["weights"] / g["weights"].sum()
    gm.means_ = g["means"]
    gm.covariances_ = g["covs"]
    gm.precisions_cholesky_ = np.stack([np.linalg.cholesky(np.linalg.inv(C)) for C in g["covs"]])
    P = gm.predict_proba(X.T)
    pv, pi = rg.memberships(X, g)
    np.testing.assert_allclose(pv, P[:, 0], atol=1e-13)
    np.testing.assert_allclose(pi, P[:, 1], atol=1e-13)


def test_membership_special_cases():
    rng = np.random.default_rng(18)
    X = rng.normal(size=(3, 20))
    C = np.diag([1.0, 2.0, 0.5])
    # identical components: the posterior is the normalised weights
    pv, pi = rg.memberships(X, _gmm(w=(0.3, 0.9), means=((1, 2, 3), (1, 2, 3)), covs=(C, C), viscous=1))
    np.testing.assert_allclose(pv, 0.75, rtol=1e-14)
    np.testing.assert_allclose(pi, 0.25, rtol=1e-14)
    # the midpoint of two equal, equally weighted components
    g = _gmm(means=((1, 0, 0), (-1, 0, 0)), covs=(C, C))
    pv, pi = rg.memberships(np.zeros((3, 1)), g)
    assert abs(pv[0] - 0.5) < 1e-15 and abs(pi[0] - 0.5) < 1e-15
    # exchanging which component is viscous exchanges the memberships
    g0 = _random_gmm(rng, viscous=0)
    g1 = dict(g0, viscous=1)
    a0, b0 = rg.memberships(X, g0)
    a1, b1 = rg.memberships(X, g1)
    np.testing.assert_array_equal(a0, b1)
    np.testing.assert_array_equal(b0, a1)
    np.testing.assert_allclose(a0 + b0, 1.0, rtol=1e-14)
    # features far in the tails of both components (densities below the FP64 range)
    pv, pi = rg.memberships(np.array([[1e6], [-3e5], [2e6]]), _random_gmm(rng))
    assert np.isfinite(pv[0]) and np.isfinite(pi[0]) and abs(pv[0] + pi[0] - 1) < 1e-15


def test_element_means_by_brute_force_on_a_tiny_element():
    st = pytest.importorskip("scipy.stats")
    # one affine element at order 1 (8 nodes), a field whose gradient varies inside it
    desc = _open_box(1, _affine_warp())
    M = _mesh(desc, 1)
    xyz = M.node_coords()
    q = np.zeros((4, M.total))
    q[1] = np.sin(1.3 * xyz[1]) + 0.2 * xyz[2]
    q[2] = xyz[0] * xyz[2]
    q[3] = np.cos(xyz[0] + 2 * xyz[1])
    # features at the 8 nodes: Q_S in [-2, -0.2], R_S in [-0.06, 0.13], Q_Omega in [1, 1.9]
    g = _gmm(means=((-0.5, 0, 1.1), (-1.5, 0.05, 1.5)), covs=(np.diag([0.3, 0.01, 0.1]), np.diag([0.3, 0.01, 0.1])))
    out = rg.detect_regions(M, q, g)
    G = rg.element_velocity_gradient(M, q, 0)
    pvs, pis = [], []
    for p in range(8):
        Gp = [[G[c, k, p] for k in range(3)] for c in range(3)]
        S = [[0.5 * (Gp[i][j] + Gp[j][i]) for j in range(3)] for i in range(3)]
        W = [[0.5 * (Gp[i][j] - Gp[j][i]) for j in range(3)] for i in range(3)]
        trS = S[0][0] + S[1][1] + S[2][2]
        trS2 = sum(S[i][j] * S[j][i] for i in range(3) for j in range(3))
        det = (S[0][0] * (S[1][1] * S[2][2] - S[1][2] * S[2][1]) - S[0][1] * (S[1][0] * S[2][2] - S[1][2] * S[2][0])
               + S[0][2] * (S[1][0] * S[2][1] - S[1][1] * S[2][0]))
        trW2 = sum(W[i][j] * W[j][i] for i in range(3) for j in range(3))
        x = [0.5 * (trS * trS - trS2), -det / 3.0, -0.5 * trW2]
        dens = [g["weights"][k] * st.multivariate_normal(g["means"][k], g["covs"][k]).pdf(x) for k in range(2)]
        pvs.append(dens[1] / (dens[0] + dens[1]))
        pis.append(dens[0] / (dens[0] + dens[1]))
        np.testing.assert_allclose(out["features"][:, p], x, atol=1e-14)
    assert abs(out["pbar"][0, 0] - math.fsum(pvs) / 8) < 1e-14
    assert abs(out["pbar"][1, 0] - math.fsum(pis) / 8) < 1e-14
    assert out["flags"][0] == (1 if math.fsum(pvs) >= math.fsum(pis) else 0)
    assert 0.05 < out["pbar"][0, 0] < 0.95  # a case where both regions carry weight


def test_a_tie_goes_to_the_viscous_region():
    w = wl.tgv_4x4x4_n3(n_elem_dir=3, order=2)
    M = orc.Mesh(w.mesh.hex, w.mesh.geom, w.mesh.geom_degree, w.orders, w.flags, orc.params())
    q = w.state(M.node_coords())
    C = np.diag([1.0, 1.0, 1.0])
    out = rg.detect_regions(M, q, _gmm(means=((0, 0, 0), (0, 0, 0)), covs=(C, C)))
    assert np.all(out["pbar"][0] == out["pbar"][1]) and np.abs(out["pbar"] - 0.5).max() < 1e-15
    assert np.all(out["flags"] == 1)


def test_the_wake_shear_layer_is_viscous_and_the_far_field_inviscid():
    # u = 1 - 0.5 exp(-r^2 / 0.25) about the line y = z = 2: a shear layer around r = 0.35
    # (Q_S = -|grad u|^2 / 4, R_S = 0, Q_Omega = |grad u|^2 / 4), zero gradient far out
    w = wl.wake_16x16x16_n4(n=16, order=3)
    M = orc.Mesh(w.mesh.hex, w.mesh.geom, w.mesh.geom_degree, w.orders, w.flags, orc.params(), w.mesh.bc_tag)
    xyz = M.node_coords()
    r2 = (xyz[1] - 2) ** 2 + (xyz[2] - 2) ** 2
    q = np.zeros((4, M.total))
    q[1] = 1 - 0.5 * np.exp(-r2 / 0.25)
    c = w.mesh.centers
    rc = np.hypot(c[:, 1] - 2, c[:, 2] - 2)
    sel = np.flatnonzero((c[:, 0] < 1.0) & ((rc < 0.6) | (rc > 1.6)))
    out = rg.detect_regions(M, q, _gmm(), elements=sel)
    near, far = rc[sel] < 0.6, rc[sel] > 1.6
    assert np.all(out["flags"][near] == 1) and np.all(out["flags"][far] == 0)
    assert np.all(np.abs(out["features"][1]) < 1e-12)  # R_S = 0 for a unidirectional shear
    np.testing.assert_allclose(out["features"][0], -out["features"][2], atol=1e-12)


def test_bad_mixtures_are_rejected():
    C = np.eye(3)
    with pytest.raises(ValueError):
        rg.memberships(np.zeros((3, 1)), _gmm(w=(0.0, 1.0), covs=(C, C)))
    with pytest.raises(ValueError):
        rg.memberships(np.zeros((3, 1)), _gmm(covs=(C, np.diag([1.0, -1.0, 1.0]))))
    with pytest.raises(ValueError):
        rg.memberships(np.zeros((3, 1)), _gmm(covs=(C, np.array([[1, 0.5, 0], [0, 1, 0], [0, 0, 1.0]]))))
    with pytest.raises(ValueError):
        rg.memberships(np.zeros((3, 1)), _gmm(covs=(C, C), viscous=2))
