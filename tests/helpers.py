"""Shared test helpers: build the oracle and the CUDA solver for one workload, same inputs."""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import oracle as orc
from paper_2403_05463_gb300 import workloads as wl


# arithmetic options of the library that do not change what the residual is
GPU_ONLY = ("fp64_divergence",)


def oracle_mesh(w: wl.Workload, params=None):
    m = w.mesh
    prm = {k: v for k, v in (params or w.params).items() if k not in GPU_ONLY}
    return orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, orc.params(**prm), m.bc_tag)


def gpu_solver(w: wl.Workload, precision=0, params=None):
    from paper_2403_05463_gb300 import dg
    return dg.Solver.from_workload(w, precision=precision, params=params)


def oracle_state(w: wl.Workload, M: orc.Mesh):
    """Initial state from the oracle's node coordinates (the CUDA path never produces inputs)."""
    return w.state(M.node_coords())


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def small_mixed(w, seed, orders=None, flags_p=0.5):
    """Copy of a workload with seeded per-element orders (in `orders`) and random flags."""
    rng = np.random.default_rng(seed)
    E = w.n_elem
    o = w.orders if orders is None else rng.integers(orders[0], orders[1] + 1, size=E).astype(np.int8)
    f = (rng.uniform(size=E) < flags_p).astype(np.uint8)
    return dataclasses.replace(w, orders=o.astype(np.int8), flags=f)
