"""ctypes binding of the FP64 CPU oracle (``dg_oracle.c``).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module. It never imports the product package and the
product never imports it.

The oracle evaluates the residual of the flagged Euler / NS-LES DGSEM of arXiv 2403.05463
(Sec. 2.3, App. A, App. B) in plain FP64, weak form, element by element.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dg_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
LIB_PATH_EXT = os.path.join(BUILD_DIR, "liboracle_ext.so")

_lock = threading.Lock()
_libs = {}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2): the FP64 library and the extended-precision
    one (long double; only for checks whose FP64 conditioning is too poor). Returns the FP64
    library path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    for path, extra in ((LIB_PATH, []), (LIB_PATH_EXT, ["-DOR_EXTENDED=1"])):
        stale = (not os.path.exists(path)) or os.path.getmtime(path) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "dg_oracle.h")))
        if force or stale:
            tmp = path + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE", *extra,
                   "-o", tmp, SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, path)
    return LIB_PATH


_P = ctypes.POINTER
_i64 = _P(ctypes.c_int64)
_i8 = _P(ctypes.c_int8)
_u8 = _P(ctypes.c_uint8)


def _params_type(real):
    class P(ctypes.Structure):
        _fields_ = [("nu", real), ("c0sq", real), ("cs", real), ("cv", real), ("closure", ctypes.c_int),
                    ("riemann", ctypes.c_int), ("mixed_face", ctypes.c_int), ("split", ctypes.c_int),
                    ("inflow", real * 4), ("gamma", real), ("prandtl", real), ("prandtl_t", real),
                    ("nodes", ctypes.c_int), ("p_inf", real)]
    return P


Params = _params_type(ctypes.c_double)
ParamsExt = _params_type(ctypes.c_longdouble)
_d = _P(ctypes.c_double)


def lib(extended: bool = False):
    with _lock:
        if extended not in _libs:
            build()
            real = ctypes.c_longdouble if extended else ctypes.c_double
            Pt = ParamsExt if extended else Params
            _d = _P(real)
            L = ctypes.CDLL(LIB_PATH_EXT if extended else LIB_PATH)
            L.or_lgl.argtypes = [ctypes.c_int, _d, _d]
            L.or_gl.argtypes = [ctypes.c_int, _d, _d]
            L.or_dmat.argtypes = [ctypes.c_int, _d]
            L.or_dmat_gl.argtypes = [ctypes.c_int, _d]
            L.or_interp_lgl.argtypes = [ctypes.c_int, ctypes.c_int, _d]
            L.or_project_lgl.argtypes = [ctypes.c_int, ctypes.c_int, _d]
            L.or_interp_gl.argtypes = [ctypes.c_int, ctypes.c_int, _d]
            L.or_project_gl.argtypes = [ctypes.c_int, ctypes.c_int, _d]
            L.or_normal_flux.argtypes = [_d, _d, real, _d]
            L.or_normal_flux.restype = None
            L.or_kep_flux.argtypes = [_d, _d, _d, _d, real, _d]
            L.or_kep_flux.restype = None
            L.or_flux_jacobian.argtypes = [_d, _d, real, _d]
            L.or_flux_jacobian.restype = None
            L.or_abs_jacobian.argtypes = [_d, _d, real, _d]
            L.or_riemann.argtypes = [_d, _d, _d, _P(Pt), _d]
            L.or_eddy_viscosity.argtypes = [_d, real, _P(Pt)]
            L.or_eddy_viscosity.restype = real
            L.or_rk3_linear.argtypes = [real]
            L.or_rk3_linear.restype = real
            L.or_create.argtypes = [ctypes.c_int64, _i64, ctypes.c_int, _d, _i8, _i8, _u8, _P(Pt)]
            L.or_create.restype = ctypes.c_void_p
            L.or_destroy.argtypes = [ctypes.c_void_p]
            L.or_destroy.restype = None
            L.or_error.restype = ctypes.c_char_p
            L.or_total_nodes.argtypes = [ctypes.c_void_p]
            L.or_total_nodes.restype = ctypes.c_int64
            L.or_offsets.argtypes = [ctypes.c_void_p]
            L.or_offsets.restype = _i64
            L.or_node_coords.argtypes = [ctypes.c_void_p, _d]
            L.or_set_visc_scale.argtypes = [ctypes.c_void_p, _d]
            L.or_element_geometry.argtypes = [ctypes.c_void_p, ctypes.c_int64, _d, _d]
            L.or_element_gradient.argtypes = [ctypes.c_void_p, _d, ctypes.c_int64, _d]
            L.or_residual.argtypes = [ctypes.c_void_p, _d, _d, ctypes.c_int64, _i64]
            L.or_rk_step.argtypes = [ctypes.c_void_p, _d, _d, real, ctypes.c_int]
            L.or_conservation.argtypes = [ctypes.c_void_p, _d, _d]
            L.or_num_threads.restype = ctypes.c_int
            L.or_set_num_threads.argtypes = [ctypes.c_int]
            L.or_set_num_threads.restype = None
            L.or_cns_flux.argtypes = [_d, _d, real, _d]
            L.or_cns_flux.restype = None
            L.or_cns_jacobian.argtypes = [_d, _d, real, _d]
            L.or_cns_jacobian.restype = None
            L.or_cns_roe_abs_jacobian.argtypes = [_d, _d, _d, real, _d]
            L.or_cns_riemann.argtypes = [_d, _d, _d, _P(Pt), _d]
            L.or_cns_element_gradient.argtypes = [ctypes.c_void_p, _d, ctypes.c_int64, _d]
            L.or_cns_residual.argtypes = [ctypes.c_void_p, _d, _d, ctypes.c_int64, _i64]
            L.or_cns_rk_step.argtypes = [ctypes.c_void_p, _d, _d, real, ctypes.c_int]
            L.or_cns_conservation.argtypes = [ctypes.c_void_p, _d, _d]
            _libs[extended] = L
    return _libs[extended]


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params(nu=0.0, c0sq=25.0, cs=0.1, cv=0.07, closure=0, riemann=0, inflow=(0.0, 1.0, 0.0, 0.0), mixed_face=0,
           split=0, gamma=1.4, prandtl=0.72, prandtl_t=0.9, nodes=0, p_inf=0.0):
    p = Params()
    p.nu, p.c0sq, p.cs, p.cv = nu, c0sq, cs, cv
    p.closure, p.riemann, p.mixed_face, p.split = closure, riemann, mixed_face, split
    p.gamma, p.prandtl, p.prandtl_t = gamma, prandtl, prandtl_t
    p.nodes = nodes
    p.p_inf = p_inf
    for i in range(4):
        p.inflow[i] = inflow[i]
    return p


# ---- 1D operators --------------------------------------------------------------------

def lgl(N):
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().or_lgl(N, _ptr(x, _d), _ptr(w, _d)):
        raise ValueError(lib().or_error().decode())
    return x, w


def gl(N):
    """Gauss-Legendre nodes and weights (N + 1 points)."""
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().or_gl(N, _ptr(x, _d), _ptr(w, _d)):
        raise ValueError(lib().or_error().decode())
    return x, w


def dmat(N):
    D = np.zeros((N + 1, N + 1))
    if lib().or_dmat(N, _ptr(D, _d)):
        raise ValueError(lib().or_error().decode())
    return D


def dmat_gl(N):
    """Derivative matrix on the N + 1 Gauss-Legendre nodes."""
    D = np.zeros((N + 1, N + 1))
    if lib().or_dmat_gl(N, _ptr(D, _d)):
        raise ValueError(lib().or_error().decode())
    return D


def interp(Ns, Nd):
    I = np.zeros((Nd + 1, Ns + 1))
    if lib().or_interp_lgl(Ns, Nd, _ptr(I, _d)):
        raise ValueError(lib().or_error().decode())
    return I


def project(Nh, Nl):
    P = np.zeros((Nl + 1, Nh + 1))
    if lib().or_project_lgl(Nh, Nl, _ptr(P, _d)):
        raise ValueError(lib().or_error().decode())
    return P


def interp_gl(Ns, Nd):
    """Interpolation from the Ns + 1 to the Nd + 1 Gauss-Legendre nodes."""
    I = np.zeros((Nd + 1, Ns + 1))
    if lib().or_interp_gl(Ns, Nd, _ptr(I, _d)):
        raise ValueError(lib().or_error().decode())
    return I


def project_gl(Nh, Nl):
    """L2 projection from degree Nh to degree Nl, both on Gauss-Legendre nodes."""
    P = np.zeros((Nl + 1, Nh + 1))
    if lib().or_project_gl(Nh, Nl, _ptr(P, _d)):
        raise ValueError(lib().or_error().decode())
    return P


def project_state(orders_old, orders_new, q_old, nodes=0):
    """The state re-laid out for new per-element orders (Sec. 3.2, re-assigning orders):
    element by element, Lagrange interpolation onto the new nodes (Gauss-Lobatto, or
    Gauss-Legendre with nodes=1) where the order grows or stays, the L2 projection (in
    reference coordinates) where it drops, applied along each of the three directions.
    q_old: [nvar][sum (N_old + 1)^3] (nvar 4, or 5 for the compressible state); returns
    [nvar][sum (N_new + 1)^3]."""
    up, down = (interp_gl, project_gl) if nodes == 1 else (interp, project)
    orders_old = np.asarray(orders_old, dtype=np.int64)
    orders_new = np.asarray(orders_new, dtype=np.int64)
    off_o = np.concatenate([[0], np.cumsum((orders_old + 1) ** 3)])
    off_n = np.concatenate([[0], np.cumsum((orders_new + 1) ** 3)])
    nv = q_old.shape[0]
    q_new = np.zeros((nv, off_n[-1]))
    ops = {}
    for e in range(len(orders_old)):
        No, Nn = int(orders_old[e]), int(orders_new[e])
        if (No, Nn) not in ops:
            ops[No, Nn] = up(No, Nn) if Nn >= No else down(No, Nn)
        T = ops[No, Nn]
        no, nn = No + 1, Nn + 1
        A = q_old[:, off_o[e]:off_o[e + 1]].reshape(nv, no, no, no)  # [v][k][j][i], i fastest
        B = np.einsum('Ia,Jb,Kc,vcba->vKJI', T, T, T, A)
        q_new[:, off_n[e]:off_n[e + 1]] = B.reshape(nv, -1)
    return q_new


# ---- pointwise -----------------------------------------------------------------------

def normal_flux(q, n, c0sq):
    out = np.zeros(4)
    lib().or_normal_flux(_ptr(_f64(q), _d), _ptr(_f64(n), _d), c0sq, _ptr(out, _d))
    return out


def kep_flux(qi, qm, ja_i, ja_m, c0sq):
    out = np.zeros(4)
    lib().or_kep_flux(_ptr(_f64(qi), _d), _ptr(_f64(qm), _d), _ptr(_f64(ja_i), _d), _ptr(_f64(ja_m), _d), c0sq,
                      _ptr(out, _d))
    return out


def flux_jacobian(q, n, c0sq):
    A = np.zeros((4, 4))
    lib().or_flux_jacobian(_ptr(_f64(q), _d), _ptr(_f64(n), _d), c0sq, _ptr(A, _d))
    return A


def abs_jacobian(q, n, c0sq):
    A = np.zeros((4, 4))
    if lib().or_abs_jacobian(_ptr(_f64(q), _d), _ptr(_f64(n), _d), c0sq, _ptr(A, _d)):
        raise ValueError(lib().or_error().decode())
    return A


def cns_flux(u, n, gamma=1.4):
    out = np.zeros(5)
    lib().or_cns_flux(_ptr(_f64(u), _d), _ptr(_f64(n), _d), gamma, _ptr(out, _d))
    return out


def cns_jacobian(u, n, gamma=1.4):
    A = np.zeros((5, 5))
    lib().or_cns_jacobian(_ptr(_f64(u), _d), _ptr(_f64(n), _d), gamma, _ptr(A, _d))
    return A


def cns_roe_abs_jacobian(uL, uR, n, gamma=1.4):
    A = np.zeros((5, 5))
    if lib().or_cns_roe_abs_jacobian(_ptr(_f64(uL), _d), _ptr(_f64(uR), _d), _ptr(_f64(n), _d), gamma, _ptr(A, _d)):
        raise ValueError("no Roe average (non-positive density or sound speed)")
    return A


def cns_riemann(uL, uR, n, prm):
    out = np.zeros(5)
    if lib().or_cns_riemann(_ptr(_f64(uL), _d), _ptr(_f64(uR), _d), _ptr(_f64(n), _d), ctypes.byref(prm), _ptr(out, _d)):
        raise ValueError("Riemann solver failed")
    return out


def riemann(qm, qp, n, prm):
    out = np.zeros(4)
    if lib().or_riemann(_ptr(_f64(qm), _d), _ptr(_f64(qp), _d), _ptr(_f64(n), _d), ctypes.byref(prm),
                        _ptr(out, _d)):
        raise ValueError(lib().or_error().decode())
    return out


def eddy_viscosity(G, delta, prm):
    return lib().or_eddy_viscosity(_ptr(_f64(np.asarray(G).reshape(9)), _d), delta, ctypes.byref(prm))


def rk3_linear(z):
    return lib().or_rk3_linear(z)


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    lib().or_set_num_threads(int(n))


# ---- mesh ----------------------------------------------------------------------------

class Mesh:
    """Oracle discretisation of one mesh (orders, flags and parameters fixed).

    extended=True evaluates in long double (inputs are widened, results rounded to FP64);
    the default is the FP64 oracle."""

    def __init__(self, hex, geom_xyz, geom_degree, orders, flags, prm, bc_tag=None, extended=False):
        self.extended = bool(extended)
        L = self._L = lib(self.extended)
        self._real = np.longdouble if self.extended else np.float64
        self._ptr_t = _P(ctypes.c_longdouble if self.extended else ctypes.c_double)
        if self.extended:
            p2 = ParamsExt()
            for name, _ in Params._fields_:
                v = getattr(prm, name)
                if name == "inflow":
                    for i in range(4):
                        p2.inflow[i] = v[i]
                else:
                    setattr(p2, name, v)
            prm = p2
        self.hex = np.ascontiguousarray(hex, dtype=np.int64)
        self.ne = self.hex.shape[0]
        gx = self._r(geom_xyz)
        orders = np.ascontiguousarray(orders, dtype=np.int8)
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        bc = None if bc_tag is None else np.ascontiguousarray(bc_tag, dtype=np.int8)
        self.prm = prm
        self.orders = orders.copy()
        self.flags = flags.copy()
        h = L.or_create(self.ne, _ptr(self.hex, _i64), geom_degree, _ptr(gx, self._ptr_t),
                        None if bc is None else _ptr(bc, _i8), _ptr(orders, _i8), _ptr(flags, _u8),
                        ctypes.byref(prm))
        if not h:
            raise ValueError(L.or_error().decode())
        self.h = h
        self.total = L.or_total_nodes(h)
        offp = L.or_offsets(h)
        self.offsets = np.ctypeslib.as_array(offp, shape=(self.ne + 1,)).copy()

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._L.or_destroy(h)
            self.h = None

    def _r(self, a):
        return np.ascontiguousarray(a, dtype=self._real)

    def node_coords(self):
        xyz = np.zeros((3, self.total), dtype=self._real)
        self._L.or_node_coords(self.h, _ptr(xyz, self._ptr_t))
        return xyz.astype(np.float64)

    def set_visc_scale(self, scale):
        s = None if scale is None else self._r(scale)
        self._L.or_set_visc_scale(self.h, None if s is None else _ptr(s, self._ptr_t))

    def element_geometry(self, e):
        n = int(self.orders[e]) + 1
        J = np.zeros(n ** 3, dtype=self._real)
        Ja = np.zeros((3, 3, n ** 3), dtype=self._real)
        self._L.or_element_geometry(self.h, e, _ptr(J, self._ptr_t), _ptr(Ja, self._ptr_t))
        return J.astype(np.float64), Ja.astype(np.float64)

    def element_gradient(self, q, e):
        n = int(self.orders[e]) + 1
        G = np.zeros((3, 3, n ** 3), dtype=self._real)
        q = self._r(q)
        self._L.or_element_gradient(self.h, _ptr(q, self._ptr_t), e, _ptr(G, self._ptr_t))
        return G.astype(np.float64)

    def residual(self, q, sel=None, out=None):
        q = self._r(q)
        assert q.shape == (4, self.total)
        R = np.zeros((4, self.total), dtype=self._real)
        if sel is None:
            rc = self._L.or_residual(self.h, _ptr(q, self._ptr_t), _ptr(R, self._ptr_t), 0, None)
        else:
            s = np.ascontiguousarray(sel, dtype=np.int64)
            rc = self._L.or_residual(self.h, _ptr(q, self._ptr_t), _ptr(R, self._ptr_t), s.size, _ptr(s, _i64))
        if rc:
            raise RuntimeError(self._L.or_error().decode())
        if out is None:
            return R.astype(np.float64)
        if sel is None:
            out[...] = R
        else:
            idx = np.concatenate([np.arange(self.offsets[e], self.offsets[e + 1]) for e in np.asarray(sel)])
            out[:, idx] = R[:, idx]
        return out

    def rk_step(self, q, g, dt, nsteps=1):
        """In place on FP64 arrays q, g (the extended oracle works on widened copies)."""
        assert q.dtype == np.float64 and g.dtype == np.float64 and q.flags.c_contiguous and g.flags.c_contiguous
        qr, gr = self._r(q), self._r(g)
        if self._L.or_rk_step(self.h, _ptr(qr, self._ptr_t), _ptr(gr, self._ptr_t), dt, nsteps):
            raise RuntimeError(self._L.or_error().decode())
        if self.extended:
            q[...] = qr
            g[...] = gr

    def conservation(self, R):
        out = np.zeros(4, dtype=self._real)
        R = self._r(R)
        self._L.or_conservation(self.h, _ptr(R, self._ptr_t), _ptr(out, self._ptr_t))
        return out.astype(np.float64)

    # ---- compressible form (App. A): state u [5][total_nodes] ------------------------------

    def cns_residual(self, u, sel=None, out=None):
        u = self._r(u)
        assert u.shape == (5, self.total)
        R = np.zeros((5, self.total), dtype=self._real)
        if sel is None:
            rc = self._L.or_cns_residual(self.h, _ptr(u, self._ptr_t), _ptr(R, self._ptr_t), 0, None)
        else:
            s = np.ascontiguousarray(sel, dtype=np.int64)
            rc = self._L.or_cns_residual(self.h, _ptr(u, self._ptr_t), _ptr(R, self._ptr_t), s.size, _ptr(s, _i64))
        if rc:
            raise RuntimeError(self._L.or_error().decode())
        if out is None:
            return R.astype(np.float64)
        idx = np.concatenate([np.arange(self.offsets[e], self.offsets[e + 1]) for e in np.asarray(sel)])
        out[:, idx] = R[:, idx]
        return out

    def cns_rk_step(self, u, g, dt, nsteps=1):
        """In place on FP64 arrays u, g [5][total_nodes]."""
        assert u.dtype == np.float64 and g.dtype == np.float64 and u.flags.c_contiguous and g.flags.c_contiguous
        ur, gr = self._r(u), self._r(g)
        if self._L.or_cns_rk_step(self.h, _ptr(ur, self._ptr_t), _ptr(gr, self._ptr_t), dt, nsteps):
            raise RuntimeError(self._L.or_error().decode())
        if self.extended:
            u[...] = ur
            g[...] = gr

    def cns_conservation(self, R):
        out = np.zeros(5, dtype=self._real)
        R = self._r(R)
        self._L.or_cns_conservation(self.h, _ptr(R, self._ptr_t), _ptr(out, self._ptr_t))
        return out.astype(np.float64)

    def cns_element_gradient(self, u, e):
        n = int(self.orders[e]) + 1
        G = np.zeros((4, 3, n ** 3), dtype=self._real)
        if self._L.or_cns_element_gradient(self.h, _ptr(self._r(u), self._ptr_t), e, _ptr(G, self._ptr_t)):
            raise RuntimeError(self._L.or_error().decode())
        return G.astype(np.float64)

    def element_nodes(self, e):
        return slice(int(self.offsets[e]), int(self.offsets[e + 1]))
