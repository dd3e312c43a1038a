"""ctypes binding of libdgflag.so (include/dg.h): argument marshalling only.

Every step of the residual and of the Runge-Kutta update runs in the library's CUDA
kernels; PyTorch only provides device memory and streams. There is no fallback: if the
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdgflag.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dg.h")

DG_OK = 0
STATUS = {0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_MESH", 3: "DG_ERR_CUDA", 4: "DG_ERR_OOM",
          5: "DG_ERR_UNSUPPORTED", 6: "DG_ERR_STATE", 7: "DG_ERR_TIMEOUT", 8: "DG_ERR_DEVICE"}

PRECISION = {"fp64": 0, "fp32": 1, "tf32x3": 2, "tf32": 3}


class DGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("hex", ctypes.POINTER(ctypes.c_int64)),
                ("geom_degree", ctypes.c_int), ("geom_xyz", ctypes.POINTER(ctypes.c_double)),
                ("bc_tag", ctypes.POINTER(ctypes.c_int8))]


class Params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("c0sq", ctypes.c_double), ("cs", ctypes.c_double),
                ("cv", ctypes.c_double), ("closure", ctypes.c_int), ("riemann", ctypes.c_int),
                ("precision", ctypes.c_int), ("mixed_face", ctypes.c_int), ("split", ctypes.c_int),
                ("model", ctypes.c_int), ("inflow", ctypes.c_double * 4), ("gamma", ctypes.c_double),
                ("prandtl", ctypes.c_double), ("prandtl_t", ctypes.c_double), ("nodes", ctypes.c_int),
                ("fp64_divergence", ctypes.c_int), ("p_inf", ctypes.c_double)]


class GMM(ctypes.Structure):
    """Two-component Gaussian mixture on the node features (Q_S, R_S, Q_Omega) (dg_gmm)."""
    _fields_ = [("weight", ctypes.c_double * 2), ("mean", (ctypes.c_double * 3) * 2),
                ("cov", ((ctypes.c_double * 3) * 3) * 2), ("viscous", ctypes.c_int), ("precision", ctypes.c_int)]


def make_gmm(weights, means, covs, viscous, precision=0) -> GMM:
    out = GMM()
    for k in range(2):
        out.weight[k] = float(weights[k])
        for i in range(3):
            out.mean[k][i] = float(means[k][i])
            for j in range(3):
                out.cov[k][i][j] = float(covs[k][i][j])
    out.viscous = int(viscous)
    out.precision = int(precision)
    return out


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)


def header_symbols():
    """Names of the functions include/dg.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_]+)\s*\(", text)))


def load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.dg_create_mesh.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(Params), ctypes.c_int,
                                     ctypes.POINTER(_vp)]
        L.dg_set_orders.argtypes = [_vp, ctypes.POINTER(ctypes.c_int8)]
        L.dg_set_element_flags.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint8)]
        L.dg_set_params.argtypes = [_vp, ctypes.POINTER(Params)]
        L.dg_get_layout.argtypes = [_vp, _i64p, ctypes.POINTER(_i64p)]
        L.dg_node_coords.argtypes = [_vp, _vp, _vp]
        L.dg_residual.argtypes = [_vp, _vp, _vp, _vp]
        L.dg_rk_step.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp]
        L.dg_residual_host.argtypes = [_vp, _vp, _vp, _vp]
        L.dg_rk_step_host.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp]
        L.dg_conservation.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_double), _vp]
        L.dg_conservation_noalloc.argtypes = [_vp, _vp, _vp, _vp]
        L.dg_autotune.argtypes = [_vp, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int]
        L.dg_project_state.argtypes = [_vp, _vp, _vp, _vp]
        L.dg_detect_regions.argtypes = [_vp, _vp, ctypes.POINTER(GMM), _vp, _vp, _vp, _vp]
        L.dg_check_device.argtypes = [_vp, _vp]
        L.dg_set_wait_limit.argtypes = [_vp, ctypes.c_int64, ctypes.c_int]
        L.dg_set_launch_overlap.argtypes = [_vp, ctypes.c_int]
        L.dg_phase_times.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp]
        L.dg_phase_bytes.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
        L.dg_launches_per_residual.argtypes = [_vp]
        L.dg_launches_per_step.argtypes = [_vp]
        L.dg_launches_per_chained_step.argtypes = [_vp]
        L.dg_last_error.restype = ctypes.c_char_p
        L.dg_destroy.argtypes = [_vp]
        L.dg_destroy.restype = None
        for name in header_symbols():
            if name not in ("dg_last_error", "dg_destroy") and not name.startswith("dg_launches"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(status):
    if status != DG_OK:
        raise DGError(status, load().dg_last_error().decode())


def make_params(p: dict, precision=0) -> Params:
    out = Params()
    out.nu, out.c0sq, out.cs, out.cv = p["nu"], p["c0sq"], p["cs"], p["cv"]
    out.closure, out.riemann = int(p.get("closure", 0)), int(p.get("riemann", 0))
    out.precision = PRECISION.get(precision, precision) if isinstance(precision, str) else int(precision)
    out.mixed_face = int(p.get("mixed_face", 0))
    out.split = int(p.get("split", 0))
    out.model = int(p.get("model", 0))
    out.gamma = float(p.get("gamma", 1.4))
    out.prandtl = float(p.get("prandtl", 0.72))
    out.prandtl_t = float(p.get("prandtl_t", 0.9))
    out.nodes = int(p.get("nodes", 0))
    out.fp64_divergence = int(p.get("fp64_divergence", 0))
    out.p_inf = float(p.get("p_inf", 0.0))
    for i, v in enumerate(p.get("inflow", (0.0, 1.0, 0.0, 0.0))):
        out.inflow[i] = v
    return out


def _stream_handle(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name, device=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on {t.device}, the mesh on cuda:{device}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One mesh on one GPU: orders, flags and parameters can be changed in place."""

    def __init__(self, hex, geom, geom_degree, params: dict, orders=None, flags=None, bc_tag=None,
                 precision=0, device=0):
        L = load()
        self._hex = np.ascontiguousarray(hex, dtype=np.int64)
        self._geom = np.ascontiguousarray(geom, dtype=np.float64)
        self._bc = None if bc_tag is None else np.ascontiguousarray(bc_tag, dtype=np.int8)
        d = MeshDesc()
        d.n_elem = self._hex.shape[0]
        d.hex = self._hex.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.geom_degree = int(geom_degree)
        d.geom_xyz = self._geom.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.bc_tag = None if self._bc is None else self._bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
        self.params = dict(params)
        self.precision = precision
        self._prm = make_params(self.params, precision)
        h = ctypes.c_void_p()
        _check(L.dg_create_mesh(ctypes.byref(d), ctypes.byref(self._prm), int(device), ctypes.byref(h)))
        self.h = h
        self.device = device
        self.n_elem = d.n_elem
        if orders is not None:
            self.set_orders(orders)
        if flags is not None:
            self.set_flags(flags)

    @classmethod
    def from_workload(cls, w, precision=0, device=0, params=None):
        m = w.mesh
        return cls(m.hex, m.geom, m.geom_degree, params or w.params, w.orders, w.flags, m.bc_tag,
                   precision=precision, device=device)

    def close(self):
        if getattr(self, "h", None):
            load().dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- configuration ----------------------------------------------------------------
    def set_orders(self, orders):
        o = np.ascontiguousarray(orders, dtype=np.int8)
        assert o.size == self.n_elem
        before = self.total_nodes
        _check(load().dg_set_orders(self.h, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))))
        self._total_before_orders = before  # the layout project_state reads q_old in

    def set_flags(self, flags):
        f = np.ascontiguousarray(flags, dtype=np.uint8)
        assert f.size == self.n_elem
        _check(load().dg_set_element_flags(self.h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))

    def set_params(self, params: dict = None, precision=None):
        if params is not None:
            self.params = dict(params)
        if precision is not None:
            self.precision = precision
        self._prm = make_params(self.params, self.precision)
        _check(load().dg_set_params(self.h, ctypes.byref(self._prm)))

    @property
    def nvar(self) -> int:
        """Planes of the state: 4 (incompressible), 5 (compressible, params["model"] = 1)."""
        return 5 if int(self.params.get("model", 0)) == 1 else 4

    def _check_state(self, t, name):
        if t.numel() != self.nvar * self.total_nodes:
            raise ValueError(f"{name} must hold [{self.nvar}][{self.total_nodes}] values")

    @property
    def total_nodes(self) -> int:
        t = ctypes.c_int64()
        _check(load().dg_get_layout(self.h, ctypes.byref(t), None))
        return t.value

    @property
    def offsets(self) -> np.ndarray:
        t = ctypes.c_int64()
        p = _i64p()
        _check(load().dg_get_layout(self.h, ctypes.byref(t), ctypes.byref(p)))
        return np.ctypeslib.as_array(p, shape=(self.n_elem + 1,)).copy()

    # ---- compute ----------------------------------------------------------------------
    def node_coords(self):
        import torch
        xyz = torch.empty((3, self.total_nodes), dtype=torch.float64, device=f"cuda:{self.device}")
        _check(load().dg_node_coords(self.h, _dev_ptr(xyz, "xyz", self.device), _stream_handle(None)))
        return xyz

    def residual(self, q, R=None, stream=None):
        import torch
        self._check_state(q, "q")
        if R is None:
            R = torch.empty_like(q)
        self._check_state(R, "R")
        _check(load().dg_residual(self.h, _dev_ptr(q, "q", self.device), _dev_ptr(R, "R", self.device),
                                  _stream_handle(stream)))
        return R

    def rk_step(self, q, g, dt, nsteps=1, t=0.0, stream=None):
        self._check_state(q, "q")
        self._check_state(g, "g")
        _check(load().dg_rk_step(self.h, _dev_ptr(q, "q", self.device), _dev_ptr(g, "g", self.device), float(t),
                                 float(dt), int(nsteps), _stream_handle(stream)))

    def residual_host(self, q, R, stream=None):
        """q, R: host arrays (numpy or pinned CPU tensors), float64 [nvar][total]."""
        self._check_state(_as_sized(q), "q")
        self._check_state(_as_sized(R), "R")
        _check(load().dg_residual_host(self.h, _host_ptr(q), _host_ptr(R), _stream_handle(stream)))

    def rk_step_host(self, q, g=None, dt=0.0, nsteps=1, t=0.0, stream=None):
        """q (and g unless None, see dg_rk_step_host): host arrays, float64 [nvar][total]."""
        self._check_state(_as_sized(q), "q")
        if g is not None:
            self._check_state(_as_sized(g), "g")
        _check(load().dg_rk_step_host(self.h, _host_ptr(q), None if g is None else _host_ptr(g), float(t), float(dt),
                                      int(nsteps), _stream_handle(stream)))

    def conservation(self, R, stream=None):
        self._check_state(R, "R")
        out = (ctypes.c_double * 5)()
        _check(load().dg_conservation(self.h, _dev_ptr(R, "R", self.device), out, _stream_handle(stream)))
        return np.array(list(out)[:self.nvar])

    def conservation_noalloc(self, R, out, stream=None):
        """The same sums into `out` (a caller-owned float64 CUDA tensor of 4 values), without
        any allocation, host copy or synchronisation; calls whose kernels overlap on one device
        race on the library's shared scratch."""
        self._check_state(R, "R")
        if out.numel() < 4:
            raise ValueError("out must hold 4 float64 values")
        _check(load().dg_conservation_noalloc(self.h, _dev_ptr(R, "R", self.device), _dev_ptr(out, "out", self.device),
                                              _stream_handle(stream)))

    def project_state(self, q_old, stream=None):
        """q_old in the layout before the last set_orders -> a new tensor in the current one
        (see dg_project_state)."""
        import torch
        before = getattr(self, "_total_before_orders", None)
        if before is None:
            raise DGError(6, "project_state: no set_orders before it")
        if q_old.numel() != self.nvar * before:
            raise ValueError(f"q_old must hold [{self.nvar}][{before}] values (the layout before the last set_orders)")
        q_new = torch.empty((self.nvar, self.total_nodes), dtype=torch.float64, device=q_old.device)
        _check(load().dg_project_state(self.h, _dev_ptr(q_old, "q_old", self.device),
                                       _dev_ptr(q_new, "q_new", self.device),
                                       _stream_handle(stream)))
        return q_new

    def detect_regions(self, q, gmm, flags=True, pbar=True, features=False, precision=None, stream=None):
        """Viscous/inviscid region detection from the state q (see dg_detect_regions). gmm is a
        GMM or a dict with weights, means, covs, viscous; precision (0 FP64, 1 FP32) overrides
        the mixture's. Returns (flags, pbar, features): uint8 [n_elem], float64 [2][n_elem],
        float64 [4][total_nodes] CUDA tensors, None where not requested. The context's own
        flags are left as they are."""
        import torch
        if isinstance(gmm, dict):
            gmm = make_gmm(gmm["weights"], gmm["means"], gmm["covs"], gmm["viscous"], gmm.get("precision", 0))
        if precision is not None:
            gmm = make_gmm(list(gmm.weight), [list(m) for m in gmm.mean], [[list(r) for r in c] for c in gmm.cov],
                           gmm.viscous, precision)
        dev = q.device
        f = torch.empty(self.n_elem, dtype=torch.uint8, device=dev) if flags else None
        pb = torch.empty((2, self.n_elem), dtype=torch.float64, device=dev) if pbar else None
        ft = torch.empty((4, self.total_nodes), dtype=torch.float64, device=dev) if features else None
        _check(load().dg_detect_regions(self.h, _dev_ptr(q, "q", self.device), ctypes.byref(gmm),
                                        None if f is None else ctypes.c_void_p(f.data_ptr()),
                                        None if pb is None else _dev_ptr(pb, "pbar", self.device),
                                        None if ft is None else _dev_ptr(ft, "features", self.device),
                                        _stream_handle(stream)))
        return f, pb, ft

    def autotune(self, cache_path=None):
        """Time the candidate launch shapes of the reduced-precision passes on this mesh and
        keep the fastest (see dg_autotune); returns the library's report."""
        buf = ctypes.create_string_buffer(8192)
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(load().dg_autotune(self.h, path, buf, len(buf)))
        return buf.value.decode()

    PHASES = ("traces", "mortar_lift", "viscous", "mortar_flux", "inviscid_update")

    def phase_times(self, q, g, dt, reps=3, stream=None):
        """Mean milliseconds per phase over `reps` RK stages (advances q, g)."""
        out = (ctypes.c_double * 5)()
        _check(load().dg_phase_times(self.h, _dev_ptr(q, "q", self.device), _dev_ptr(g, "g", self.device), float(dt),
                                     int(reps), out, _stream_handle(stream)))
        return dict(zip(self.PHASES, list(out)))

    def phase_bytes(self):
        out = (ctypes.c_double * 5)()
        _check(load().dg_phase_bytes(self.h, out))
        return dict(zip(self.PHASES, list(out)))

    def set_wait_limit(self, polls=0, stop_tile=-1):
        """Poll budget of the bounded device-side waits (0: the default) and the stop-tile test
        hook (-1: off); see dg_set_wait_limit."""
        _check(load().dg_set_wait_limit(self.h, int(polls), int(stop_tile)))

    def set_launch_overlap(self, enable=True):
        """Overlapped (programmatic-serialisation) launches of the pipelined passes, on by
        default; off gives plain launches with identical results. See dg_set_launch_overlap."""
        _check(load().dg_set_launch_overlap(self.h, 1 if enable else 0))

    def check_device(self, stream=None):
        _check(load().dg_check_device(self.h, _stream_handle(stream)))

    @property
    def launches_per_residual(self):
        return load().dg_launches_per_residual(self.h)

    @property
    def launches_per_step(self):
        return load().dg_launches_per_step(self.h)

    @property
    def launches_per_chained_step(self):
        """Launches of a step that follows another in the same rk_step call."""
        return load().dg_launches_per_chained_step(self.h)


class _as_sized:
    """numel() of a numpy array or a tensor, for the size checks."""
    def __init__(self, a):
        self._n = a.size if isinstance(a, np.ndarray) else a.numel()

    def numel(self):
        return self._n


def _host_ptr(a):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("host array must be C-contiguous float64")
        return ctypes.c_void_p(a.ctypes.data)
    import torch
    if isinstance(a, torch.Tensor) and not a.is_cuda and a.dtype == torch.float64 and a.is_contiguous():
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("host array must be a float64 numpy array or CPU tensor")
