"""FP64 oracle of the viscous/inviscid region detection of arXiv 2403.05463 (Sec. 2.1).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import this module. It never imports the product package and the product
never imports it.

Steps, in the order of Sec. 2.1, each written as its plain definition:
  1. velocity gradient J = grad U at every node of every element;
  2. the invariants Q_S = (tr(S)^2 - tr(S^2)) / 2, R_S = -det(S) / 3 of the strain rate
     S = (J + J^T) / 2 and Q_Omega = -tr(Omega^2) / 2 of the rotation rate Omega = (J - J^T) / 2;
  3. the two membership probabilities of each node under a given two-component Gaussian
     mixture on the features (Q_S, R_S, Q_Omega) (the E-step of the mixture: posterior of each
     component);
  4. the mean of each membership over the (P+1)^3 nodes of the element (the two equations of
     Sec. 2.1) and the region with the larger mean.

Readings where the paper is silent:
  * J is the gradient of the element's own velocity polynomial (no interface lifting), by the
    chain rule with the discrete metric terms: J_ck = (1/J) sum_d (J dxi_d/dx_k) du_c/dxi_d,
    at the mesh's nodes: Gauss-Lobatto, or the Gauss-Legendre points the paper's detection
    uses (the derivative matrix of the mesh's own node set).
  * The mixture is an input (its fitting needs developed-flow snapshots and stays outside):
    weights, means and covariances of the two components in the raw feature units, and which
    component is the viscous/rotational one. Any per-feature scaling used while fitting folds
    exactly into the means and covariances.
  * A tie of the two element means goes to the viscous region (the safe side: it keeps the
    viscous terms).
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as orc


def element_velocity_gradient(M: orc.Mesh, q, e):
    """J[c][k][node] = d u_c / d x_k of element e's velocity polynomial at its nodes (step 1)."""
    N = int(M.orders[e])
    n = N + 1
    D = orc.dmat_gl(N) if M.prm.nodes == 1 else orc.dmat(N)  # the mesh's own node set
    sl = M.element_nodes(e)
    U = np.asarray(q[1:4, sl], dtype=np.float64).reshape(3, n, n, n)  # [c][k3][k2][k1], xi_1 fastest
    dU = np.zeros((3, 3, n, n, n))  # [c][d] du_c / dxi_{d+1}
    dU[:, 0] = np.einsum('im,ckjm->ckji', D, U)
    dU[:, 1] = np.einsum('jm,ckmi->ckji', D, U)
    dU[:, 2] = np.einsum('km,cmji->ckji', D, U)
    dU = dU.reshape(3, 3, n ** 3)
    Jac, Ja = M.element_geometry(e)  # Ja[d][k] = J dxi_d / dx_k
    G = np.einsum('dkp,cdp->ckp', Ja, dU) / Jac
    return G


def invariants(G):
    """(Q_S, R_S, Q_Omega) from velocity gradients G[c][k][...] (step 2)."""
    Gm = np.moveaxis(np.asarray(G, dtype=np.float64), (0, 1), (-2, -1))  # [..., c, k]
    S = 0.5 * (Gm + np.swapaxes(Gm, -1, -2))
    W = 0.5 * (Gm - np.swapaxes(Gm, -1, -2))
    trS = np.trace(S, axis1=-2, axis2=-1)
    trS2 = np.trace(S @ S, axis1=-2, axis2=-1)
    QS = 0.5 * (trS ** 2 - trS2)
    RS = -np.linalg.det(S) / 3.0
    QW = -0.5 * np.trace(W @ W, axis1=-2, axis2=-1)
    return np.stack([QS, RS, QW])


def check_gmm(gmm):
    w = np.asarray(gmm["weights"], dtype=np.float64)
    mu = np.asarray(gmm["means"], dtype=np.float64)
    C = np.asarray(gmm["covs"], dtype=np.float64)
    if w.shape != (2,) or mu.shape != (2, 3) or C.shape != (2, 3, 3):
        raise ValueError("a two-component mixture on three features is expected")
    if not (np.all(np.isfinite(w)) and np.all(w > 0)):
        raise ValueError("mixture weights must be positive")
    for k in range(2):
        if not np.allclose(C[k], C[k].T, rtol=0, atol=1e-12 * np.abs(C[k]).max()):
            raise ValueError("covariances must be symmetric")
        if np.linalg.eigvalsh(C[k]).min() <= 0:
            raise ValueError("covariances must be positive definite")
    if gmm["viscous"] not in (0, 1):
        raise ValueError("viscous names component 0 or 1")
    return w, mu, C


def gaussian_log_density(X, mean, cov):
    """log of the 3-variate normal density at the columns of X[3][...]."""
    X = np.asarray(X, dtype=np.float64)
    d = X.reshape(3, -1) - np.asarray(mean, dtype=np.float64)[:, None]
    sign, logdet = np.linalg.slogdet(2.0 * np.pi * np.asarray(cov, dtype=np.float64))
    m = np.einsum('ip,ip->p', d, np.linalg.solve(cov, d))
    return (-0.5 * m - 0.5 * logdet).reshape(X.shape[1:])


def memberships(X, gmm):
    """Posterior probability of each component at each feature column of X[3][...] (step 3):
    p_k = w_k N(x | mu_k, C_k) / sum_j w_j N(x | mu_j, C_j), evaluated through logarithms so that
    densities far in the tails do not underflow. Returns (p_v, p_i)."""
    w, mu, C = check_gmm(gmm)
    L = np.stack([np.log(w[k]) + gaussian_log_density(X, mu[k], C[k]) for k in range(2)])
    top = L.max(axis=0)
    lse = top + np.log(np.exp(L[0] - top) + np.exp(L[1] - top))
    P = np.exp(L - lse)
    v = gmm["viscous"]
    return P[v], P[1 - v]


def detect_regions(M: orc.Mesh, q, gmm, elements=None):
    """Steps 1-4 on the elements given (all by default). Returns a dict with, per node of those
    elements (in element order), ``features`` [3][...] and ``p_v``, ``p_i``; per element,
    ``pbar`` [2][...] (mean viscous, mean inviscid membership) and ``flags`` (1 viscous/NS)."""
    elements = np.arange(M.ne) if elements is None else np.asarray(elements)
    feats, pv, pi, pbar, flags = [], [], [], [], []
    for e in elements:
        F = invariants(element_velocity_gradient(M, q, int(e)))
        a, b = memberships(F, gmm)
        feats.append(F)
        pv.append(a)
        pi.append(b)
        mv, mi = a.mean(), b.mean()  # (1/N) sum over the N = (P+1)^3 nodes
        pbar.append((mv, mi))
        flags.append(1 if mv >= mi else 0)
    return {"features": np.concatenate(feats, axis=1), "p_v": np.concatenate(pv), "p_i": np.concatenate(pi),
            "pbar": np.array(pbar).T.copy(), "flags": np.array(flags, dtype=np.uint8)}
