"""Seeded synthetic workloads: hexahedral meshes, per-element orders and flags, initial states.

This module is the one place shared by the CUDA path's tests/benchmark and the CPU oracle.
It holds no arithmetic of the discretisation: it only lays out structured hexahedral meshes
(vertex ids with periodic identification, element geometry nodes, boundary tags), draws
flags/orders and evaluates initial fields at node coordinates the caller supplies.

The five workloads stand in for the paper's NACA0012 and wind-turbine runs (Sec. 3; meshes
and experimental data are not available) with the shapes the benchmark names:
  tgv_4x4x4_n3        periodic cube [0,2pi]^3, 4^3 elements, N = 3, all NS, Taylor-Green
  wake_16x16x16_n4    box [0,8]x[0,4]^2, 16^3, N = 4, Gaussian wake, NS within r = 0.8 of the axis
  tgv_32x32x32_n5     periodic cube, 32^3, N = 5, Taylor-Green + 1% noise, 30% NS slab
  padapt_32x32x32     curved periodic unit cube (degree-2 geometry), 32^3, mixed N in 2..7
  mixed_64x64x64_n4   stretched box [0,8]x[0,4]^2, 64^3, N = 4, 25% NS, synthetic turbulence
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


# ---- counter-based random numbers (SplitMix64) ----------------------------------------

def splitmix64(x):
    """SplitMix64 finaliser on a uint64 array (Steele, Lea & Flood 2014)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def node_noise(seed: int, elem: np.ndarray, local: np.ndarray, var: int, amp: float) -> np.ndarray:
    """U(-amp, amp) keyed on (seed, element, local node, variable): independent of layout."""
    h = splitmix64(np.full(elem.shape, seed, dtype=np.uint64))
    h = splitmix64(h ^ elem.astype(np.uint64))
    h = splitmix64(h ^ local.astype(np.uint64))
    h = splitmix64(h ^ np.uint64(var))
    u = (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return amp * (2.0 * u - 1.0)


# ---- meshes -----------------------------------------------------------------------------

@dataclasses.dataclass
class MeshDesc:
    hex: np.ndarray          # [E][8] int64 vertex ids, corner c = c0 + 2 c1 + 4 c2
    geom: np.ndarray         # [E][(g+1)^3][3] float64 geometry nodes, xi_1 fastest
    geom_degree: int
    bc_tag: Optional[np.ndarray]  # [E][6] int8 (-1 interior, 1 inflow, 2 outflow) or None
    centers: np.ndarray      # [E][3] undeformed cell centres (for flag/order selection)
    shape: tuple             # (nx, ny, nz)


def box_mesh(nx, ny, nz, xb, yb, zb, periodic=(True, True, True), geom_degree=1,
             warp: Optional[Callable] = None, bc_lohi=(1, 2)) -> MeshDesc:
    """Structured hexahedral mesh with element boundaries xb, yb, zb (lengths n+1).

    Element (i, j, k) has index i + nx (j + ny k). Vertex ids wrap in periodic directions,
    so periodic faces match by their corner ids. Geometry nodes of degree 1 or 2 sit at
    the reference points {-1, 1} or {-1, 0, 1} (the Gauss-Lobatto points of those degrees);
    ``warp`` maps undeformed (x, y, z) arrays to deformed ones; ``bc_lohi`` gives the boundary
    tags of the low and high faces of every non-periodic direction.
    """
    assert geom_degree in (1, 2)
    xb, yb, zb = (np.asarray(a, dtype=np.float64) for a in (xb, yb, zb))
    nvx = nx if periodic[0] else nx + 1
    nvy = ny if periodic[1] else ny + 1
    nvz = nz if periodic[2] else nz + 1

    def vid(i, j, k):
        i = i % nx if periodic[0] else i
        j = j % ny if periodic[1] else j
        k = k % nz if periodic[2] else k
        return i + nvx * (j + nvy * k)

    E = nx * ny * nz
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    hexa = np.zeros((E, 8), dtype=np.int64)
    for c in range(8):
        c0, c1, c2 = c & 1, (c >> 1) & 1, (c >> 2) & 1
        hexa[:, c] = vid(ii + c0, jj + c1, kk + c2)
    ng = geom_degree + 1
    t = np.linspace(-1.0, 1.0, ng)
    geom = np.zeros((E, ng ** 3, 3))
    for c in range(ng):
        for b in range(ng):
            for a in range(ng):
                p = a + ng * (b + ng * c)
                x = xb[ii] + 0.5 * (t[a] + 1.0) * (xb[ii + 1] - xb[ii])
                y = yb[jj] + 0.5 * (t[b] + 1.0) * (yb[jj + 1] - yb[jj])
                z = zb[kk] + 0.5 * (t[c] + 1.0) * (zb[kk + 1] - zb[kk])
                if warp is not None:
                    x, y, z = warp(x, y, z)
                geom[:, p, 0], geom[:, p, 1], geom[:, p, 2] = x, y, z
    centers = np.stack([0.5 * (xb[ii] + xb[ii + 1]), 0.5 * (yb[jj] + yb[jj + 1]),
                        0.5 * (zb[kk] + zb[kk + 1])], axis=1)
    bc = None
    if not all(periodic):
        bc = np.full((E, 6), -1, dtype=np.int8)
        if not periodic[0]:
            bc[ii == 0, 0] = bc_lohi[0]
            bc[ii == nx - 1, 1] = bc_lohi[1]
        if not periodic[1]:
            bc[jj == 0, 2] = bc_lohi[0]
            bc[jj == ny - 1, 3] = bc_lohi[1]
        if not periodic[2]:
            bc[kk == 0, 4] = bc_lohi[0]
            bc[kk == nz - 1, 5] = bc_lohi[1]
    return MeshDesc(hexa, geom, geom_degree, bc, centers, (nx, ny, nz))


# The 24 proper rotations of the reference cube as (perm, sign): xi_old[d] = sign[d] * xi_new[perm[d]].
def _cube_rotations():
    import itertools
    rots = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            M = np.zeros((3, 3))
            for d in range(3):
                M[d, perm[d]] = signs[d]
            if round(np.linalg.det(M)) == 1:
                rots.append((perm, signs))
    return rots


CUBE_ROTATIONS = _cube_rotations()


def rotation_index_map(rot, n):
    """For a reference-cube rotation and n points per direction (symmetric node set),
    returns old_index[new_index] on the n^3 lexicographic grid."""
    perm, signs = rot
    idx = np.zeros(n ** 3, dtype=np.int64)
    for c in range(n):
        for b in range(n):
            for a in range(n):
                new = (a, b, c)
                old = [0, 0, 0]
                for d in range(3):
                    v = new[perm[d]]
                    old[d] = v if signs[d] == 1 else n - 1 - v
                idx[a + n * (b + n * c)] = old[0] + n * (old[1] + n * old[2])
    return idx


def rotate_elements(mesh: MeshDesc, seed: int):
    """Re-number every element's local frame by a seeded proper rotation of the reference
    cube (corners, geometry nodes and boundary tags move consistently). Returns the new
    mesh and the rotation chosen per element."""
    rng = np.random.default_rng(seed)
    E = mesh.hex.shape[0]
    rot_of = rng.integers(0, len(CUBE_ROTATIONS), size=E)
    ng = mesh.geom_degree + 1
    hexa = np.empty_like(mesh.hex)
    geom = np.empty_like(mesh.geom)
    bc = None if mesh.bc_tag is None else np.empty_like(mesh.bc_tag)
    for r, rot in enumerate(CUBE_ROTATIONS):
        sel = rot_of == r
        if not sel.any():
            continue
        cmap = rotation_index_map(rot, 2)
        gmap = rotation_index_map(rot, ng)
        hexa[sel] = mesh.hex[sel][:, cmap]
        geom[sel] = mesh.geom[sel][:, gmap]
        if bc is not None:
            # new face (d_new, s_new) is old face (d_old, s_old) with d_old = the direction
            # whose new-frame axis is d_new
            perm, signs = rot
            fmap = np.zeros(6, dtype=np.int64)
            for d_old in range(3):
                d_new = perm[d_old]
                for s_new in range(2):
                    s_old = s_new if signs[d_old] == 1 else 1 - s_new
                    fmap[2 * d_new + s_new] = 2 * d_old + s_old
            bc[sel] = mesh.bc_tag[sel][:, fmap]
    return MeshDesc(hexa, geom, mesh.geom_degree, bc, mesh.centers, mesh.shape), rot_of


# ---- layout helpers ---------------------------------------------------------------------

def offsets(orders: np.ndarray) -> np.ndarray:
    n3 = (orders.astype(np.int64) + 1) ** 3
    off = np.zeros(orders.size + 1, dtype=np.int64)
    np.cumsum(n3, out=off[1:])
    return off


def node_keys(orders: np.ndarray):
    """Element index and local node index of every node in the SoA layout."""
    off = offsets(orders)
    total = int(off[-1])
    n3 = np.diff(off)
    elem = np.repeat(np.arange(orders.size, dtype=np.int64), n3)
    local = np.arange(total, dtype=np.int64) - np.repeat(off[:-1], n3)
    return elem, local


# ---- initial fields -------------------------------------------------------------------

def tgv_state(xyz):
    x, y, z = xyz
    q = np.zeros((4,) + x.shape)
    q[0] = (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    q[1] = np.sin(x) * np.cos(y) * np.cos(z)
    q[2] = -np.cos(x) * np.sin(y) * np.cos(z)
    return q


def wake_velocity(y, z):
    return 1.0 - 0.5 * np.exp(-((y - 2.0) ** 2 + (z - 2.0) ** 2) / 0.25)


def shear_layer_state(xyz):
    x, y, z = xyz
    q = np.zeros((4,) + x.shape)
    q[1] = np.tanh((y - 0.5) / 0.05)
    q[2] = 0.05 * np.sin(2 * np.pi * x) * np.exp(-((y - 0.5) / 0.1) ** 2)
    q[3] = 0.02 * np.sin(2 * np.pi * z) * np.cos(2 * np.pi * x)
    return q


@dataclasses.dataclass
class FourierModes:
    k: np.ndarray      # [M][3] wave vectors on the periodic lattice
    amp: np.ndarray    # [M][3] amplitude * direction (perpendicular to k)
    phase: np.ndarray  # [M]


def kraichnan_modes(seed, lengths, nmodes=64, kmin=None, kmax=None, rms=0.05):
    """Divergence-free random Fourier modes with an E(k) ~ k^(-5/3) spectrum, |k| log-spaced
    in [kmin, kmax] and snapped to the periodic lattice, scaled to a per-component rms."""
    rng = np.random.default_rng(seed)
    L = np.asarray(lengths, dtype=np.float64)
    kmin = 2 * np.pi / L.min() if kmin is None else kmin
    kmax = kmax if kmax is not None else np.pi * 64 / L.min()
    kmag = np.exp(np.linspace(np.log(kmin), np.log(kmax), nmodes))
    dk = np.gradient(kmag)
    ks, amps = [], []
    for m in range(nmodes):
        while True:
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            kv = np.round(kmag[m] * d * L / (2 * np.pi)) * (2 * np.pi) / L
            if np.linalg.norm(kv) > 0:
                break
        r = rng.normal(size=3)
        sig = np.cross(kv, r)
        sig /= np.linalg.norm(sig)
        ks.append(kv)
        amps.append(math.sqrt(kmag[m] ** (-5.0 / 3.0) * dk[m]) * sig)
    k = np.array(ks)
    amp = np.array(amps)
    # per-component rms of sum_m a_m cos(k_m.x + phi_m): sqrt(sum |a_m|^2 / 6)
    cur = math.sqrt(float((amp ** 2).sum()) / 6.0)
    amp *= rms / cur
    phase = rng.uniform(0, 2 * np.pi, size=nmodes)
    return FourierModes(k, amp, phase)


def fourier_velocity(modes: FourierModes, xyz, chunk=1 << 22):
    """Velocity of the Fourier modes at points xyz [3][T] (numpy array or torch tensor)."""
    if hasattr(xyz, "device") and hasattr(xyz, "dtype") and not isinstance(xyz, np.ndarray):
        import torch
        k = torch.as_tensor(modes.k, dtype=xyz.dtype, device=xyz.device)
        amp = torch.as_tensor(modes.amp, dtype=xyz.dtype, device=xyz.device)
        ph = torch.as_tensor(modes.phase, dtype=xyz.dtype, device=xyz.device)
        out = torch.zeros((3, xyz.shape[1]), dtype=xyz.dtype, device=xyz.device)
        for m in range(k.shape[0]):
            out += amp[m][:, None] * torch.cos(k[m] @ xyz + ph[m])[None, :]
        return out
    x = np.asarray(xyz)
    out = np.zeros((3, x.shape[1]))
    for s in range(0, x.shape[1], chunk):
        xs = x[:, s:s + chunk]
        acc = np.zeros((3, xs.shape[1]))
        for m in range(modes.k.shape[0]):
            c = np.cos(modes.k[m] @ xs + modes.phase[m])
            acc += modes.amp[m][:, None] * c[None, :]
        out[:, s:s + chunk] = acc
    return out


# ---- workloads --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    mesh: MeshDesc
    orders: np.ndarray       # int8 [E]
    flags: np.ndarray        # uint8 [E]
    params: dict
    seed: int
    dt: float
    steps: int
    state_fn: Callable       # (xyz [3][T], elem [T], local [T]) -> q [4][T]

    @property
    def n_elem(self):
        return self.orders.size

    @property
    def total_nodes(self):
        return int(((self.orders.astype(np.int64) + 1) ** 3).sum())

    @property
    def ns_fraction(self):
        return float(self.flags.mean())

    def state(self, xyz):
        elem, local = node_keys(self.orders)
        return np.ascontiguousarray(self.state_fn(np.asarray(xyz), elem, local))

    def with_flags(self, flags):
        return dataclasses.replace(self, flags=np.ascontiguousarray(flags, dtype=np.uint8))


def default_params(**kw):
    p = dict(nu=0.0, c0sq=25.0, cs=0.1, cv=0.07, closure=0, riemann=0, inflow=(0.0, 1.0, 0.0, 0.0))
    p.update(kw)
    return p


def tgv_4x4x4_n3(n_elem_dir=4, order=3):
    """Taylor-Green vortex, periodic [0,2pi]^3, all NS + Smagorinsky (Cs 0.1), Re 1600."""
    nx = n_elem_dir
    b = np.linspace(0, 2 * np.pi, nx + 1)
    mesh = box_mesh(nx, nx, nx, b, b, b)
    E = nx ** 3
    return Workload("tgv_4x4x4_n3" if nx == 4 else f"tgv_{nx}x{nx}x{nx}_n{order}", mesh,
                    np.full(E, order, np.int8), np.ones(E, np.uint8),
                    default_params(nu=1.0 / 1600.0), 1001, 1e-3, 10,
                    lambda xyz, e, l: tgv_state(xyz))


def wake_16x16x16_n4(n=16, order=4, periodic_x=False, all_ns=False):
    """Gaussian wake deficit, box [0,8]x[0,4]^2, Re 1e4, NS within radius 0.8 of y=z=2."""
    seed = 1002
    mesh = box_mesh(n, n, n, np.linspace(0, 8, n + 1), np.linspace(0, 4, n + 1), np.linspace(0, 4, n + 1),
                    periodic=(periodic_x, True, True))
    r = np.hypot(mesh.centers[:, 1] - 2.0, mesh.centers[:, 2] - 2.0)
    flags = np.ones(n ** 3, np.uint8) if all_ns else (r < 0.8).astype(np.uint8)

    def state(xyz, e, l):
        q = np.zeros((4, xyz.shape[1]))
        q[1] = wake_velocity(xyz[1], xyz[2])
        for v in (1, 2, 3):
            q[v] += node_noise(seed, e, l, v, 0.01)
        return q

    name = f"wake_{n}x{n}x{n}_n{order}" + ("_periodic" if periodic_x else "")
    return Workload(name, mesh, np.full(n ** 3, order, np.int8), flags,
                    default_params(nu=1e-4), seed, 1e-3, 10, state)


def tgv_32x32x32_n5(n=32, order=5, ns_fraction=0.3):
    """Taylor-Green + 1% noise, periodic, 30% NS in a seeded contiguous slab (lexicographic)."""
    seed = 1003
    b = np.linspace(0, 2 * np.pi, n + 1)
    mesh = box_mesh(n, n, n, b, b, b)
    E = n ** 3
    rng = np.random.default_rng(seed)
    start = int(rng.integers(0, E))
    count = int(round(ns_fraction * E))
    flags = np.zeros(E, np.uint8)
    flags[(start + np.arange(count)) % E] = 1

    def state(xyz, e, l):
        q = tgv_state(xyz)
        for v in range(4):
            q[v] += node_noise(seed, e, l, v, 0.01)
        return q

    return Workload(f"tgv_{n}x{n}x{n}_n{order}", mesh, np.full(E, order, np.int8), flags,
                    default_params(nu=1.0 / 1600.0), seed, 1e-3, 10, state)


def padapt_32x32x32(n=32, amp=0.05):
    """Curved periodic unit cube (x_k += amp sin(2 pi x) sin(2 pi y) sin(2 pi z), degree-2
    geometry); NS + N in {6,7} in the central shear layer |y-0.5| < 0.1, Euler with
    N in {3,4,5} (weights 0.4/0.4/0.2) for 0.1 <= |y-0.5| < 0.2, Euler N in {2,3} elsewhere."""
    seed = 1004

    def warp(x, y, z):
        s = amp * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
        return x + s, y + s, z + s

    b = np.linspace(0, 1, n + 1)
    mesh = box_mesh(n, n, n, b, b, b, geom_degree=2, warp=warp)
    E = n ** 3
    rng = np.random.default_rng(seed)
    dy = np.abs(mesh.centers[:, 1] - 0.5)
    u = rng.uniform(size=E)
    orders = np.where(u < 0.5, 2, 3)
    mid = (dy >= 0.1) & (dy < 0.2)
    orders = np.where(mid, np.where(u < 0.4, 3, np.where(u < 0.8, 4, 5)), orders)
    core = dy < 0.1
    orders = np.where(core, np.where(u < 0.5, 6, 7), orders)
    flags = core.astype(np.uint8)

    def state(xyz, e, l):
        q = shear_layer_state(xyz)
        for v in (1, 2, 3):
            q[v] += node_noise(seed, e, l, v, 0.01)
        return q

    return Workload(f"padapt_{n}x{n}x{n}", mesh, orders.astype(np.int8), flags,
                    default_params(nu=1e-4), seed, 2e-4, 1, state)


def stretched_faces(n, length, ratio):
    h0 = length * (ratio - 1.0) / (ratio ** n - 1.0)
    return h0 * (ratio ** np.arange(n + 1) - 1.0) / (ratio - 1.0)


def mixed_64x64x64_n4(n=64, order=4, y_wall=0.2, r_wake=0.4, all_ns=False, all_euler=False):
    """Stretched box [0,8]x[0,4]^2 (y ratio 1.05 toward y = 0), N = 4, NS in the near-wall band
    y < y_wall and the wake band |y-2| < r, |z-2| < r (about 25%), synthetic turbulence
    (64 random Fourier modes, k^-5/3, rms 0.05) on u = 1. Periodic in all directions."""
    seed = 1005
    yb = stretched_faces(n, 4.0, 1.05)
    yb[-1] = 4.0
    mesh = box_mesh(n, n, n, np.linspace(0, 8, n + 1), yb, np.linspace(0, 4, n + 1))
    c = mesh.centers
    ns = (c[:, 1] < y_wall) | ((np.abs(c[:, 1] - 2.0) < r_wake) & (np.abs(c[:, 2] - 2.0) < r_wake))
    if all_ns:
        ns[:] = True
    if all_euler:
        ns[:] = False
    modes = kraichnan_modes(seed, (8.0, 4.0, 4.0), nmodes=64, kmin=2 * np.pi / 4.0, kmax=np.pi * n / 4.0)

    def state(xyz, e, l):
        v = fourier_velocity(modes, xyz)
        if isinstance(v, np.ndarray):
            q = np.zeros((4, v.shape[1]))
        else:
            q = v.new_zeros((4, v.shape[1]))
        q[1:] = v
        q[1] += 1.0
        return q

    name = f"mixed_{n}x{n}x{n}_n{order}"
    return Workload(name, mesh, np.full(n ** 3, order, np.int8), ns.astype(np.uint8),
                    default_params(nu=1e-4), seed, 2e-4, 100, state)


def channel_walls(n=8, order=4, wall=3, wavy=0.08):
    """Channel between walls at y = 0 and y = 2 (boundary tag 3 no-slip, 4 free-slip), periodic
    in x and z over 2 pi, Re 1e3; degree-2 geometry with wavy walls y += wavy sin x cos z; NS
    within 0.5 of either wall, Euler in the core; Poiseuille-like profile plus noise."""
    seed = 1006
    b = np.linspace(0, 2 * np.pi, n + 1)
    yb = np.linspace(0, 2, n + 1)

    def warp(x, y, z):
        return x, y + wavy * np.sin(x) * np.cos(z), z

    mesh = box_mesh(n, n, n, b, yb, b, periodic=(True, False, True), geom_degree=2, warp=warp,
                    bc_lohi=(wall, wall))
    yc = mesh.centers[:, 1]
    flags = ((yc < 0.5) | (yc > 1.5)).astype(np.uint8)

    def state(xyz, e, l):
        q = np.zeros((4, xyz.shape[1]))
        yy = xyz[1] - wavy * np.sin(xyz[0]) * np.cos(xyz[2])
        q[1] = 1.5 * yy * (2.0 - yy)
        q[2] = 0.05 * np.sin(np.pi * yy) * np.cos(xyz[0])
        q[3] = 0.05 * np.sin(np.pi * yy) * np.sin(xyz[2])
        for v in (1, 2, 3):
            q[v] += node_noise(seed, e, l, v, 0.01)
        return q

    return Workload(f"channel_{n}x{n}x{n}_n{order}_{'noslip' if wall == 3 else 'slip'}", mesh,
                    np.full(n ** 3, order, np.int8), flags, default_params(nu=1e-3), seed, 1e-3, 10, state)


def cns_state(xyz, seed, period=1.0):
    """Conservative state (rho, rho v1, rho v2, rho v3, rho e) of the compressible form for a
    mesh periodic with the given period: smooth fields with seeded phases, density 1 +- 0.2,
    velocity ~0.5 and total energy ~20, so the pressure stays positive (Mach ~0.25 at gamma
    1.4). Returns [5][T]."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2 * np.pi, 8)
    k = 2 * np.pi / period
    x, y, z = np.asarray(xyz)
    rho = 1.0 + 0.2 * np.sin(k * x + ph[0]) * np.cos(k * y + ph[1]) * np.sin(k * z + ph[2])
    v1 = 0.5 + 0.3 * np.sin(k * x + ph[3]) * np.cos(k * y)
    v2 = -0.3 * np.cos(k * x) * np.sin(k * y + ph[4]) + 0.2
    v3 = 0.2 * np.sin(k * z + ph[5]) * np.cos(k * x)
    E = 20.0 + 0.5 * np.cos(2 * k * x + ph[6]) * np.cos(k * y + ph[7])
    return np.ascontiguousarray(np.stack([rho, rho * v1, rho * v2, rho * v3, E]))


def cns_tgv(n=32, order=4, ns_fraction=0.3, curved=False):
    """Compressible form (App. A): periodic [0,2pi]^3, smooth seeded state of cns_state (Mach
    ~0.25), mu = 1/1600, Vreman (Cv 0.07), Pr 0.72, Pr_t 0.9; NS in a seeded contiguous run of
    30% of the elements (lexicographic). curved=True warps the mesh with a degree-2 geometry
    (x_k += 0.1 sin x sin y sin z)."""
    seed = 1007
    b = np.linspace(0, 2 * np.pi, n + 1)
    warp = None
    if curved:
        def warp(x, y, z):
            s = 0.1 * np.sin(x) * np.sin(y) * np.sin(z)
            return x + s, y + s, z + s
    mesh = box_mesh(n, n, n, b, b, b, geom_degree=2 if curved else 1, warp=warp)
    E = n ** 3
    rng = np.random.default_rng(seed)
    start = int(rng.integers(0, E))
    count = int(round(ns_fraction * E))
    flags = np.zeros(E, np.uint8)
    flags[(start + np.arange(count)) % E] = 1
    params = default_params(nu=1.0 / 1600.0, closure=1, model=1, gamma=1.4, prandtl=0.72, prandtl_t=0.9)
    return Workload(f"cns_tgv_{n}x{n}x{n}_n{order}" + ("_curved" if curved else ""), mesh,
                    np.full(E, order, np.int8), flags, params, seed, 5e-4, 10,
                    lambda xyz, e, l: cns_state(xyz, seed, period=2 * np.pi))


WORKLOADS = {
    "tgv_4x4x4_n3": tgv_4x4x4_n3,
    "wake_16x16x16_n4": wake_16x16x16_n4,
    "tgv_32x32x32_n5": tgv_32x32x32_n5,
    "padapt_32x32x32": padapt_32x32x32,
    "mixed_64x64x64_n4": mixed_64x64x64_n4,
    "channel_walls": channel_walls,
    "cns_tgv": cns_tgv,
}
