#!/usr/bin/env python
"""Throughput of the flagged Euler / NS-LES DGSEM Runge-Kutta step on GB300.

One benchmark step = one low-storage RK3 step = three residual evaluations + updates over the
whole mesh (every phase of the hot path: traces, viscous pass on NS elements, inviscid pass,
surface terms, FP64 update). The metric is DOF-updates/s per RK stage:
    value = n_ranks * DOF * 3 / (time per step),  DOF = sum_e (N_e + 1)^3.

Default workload: 64^3 stretched hexahedra, N = 4 (32.8 M DOF), 25% NS + Smagorinsky,
synthetic turbulence on u = 1 (the large mixed configuration). Its state (q and g: 2.1 GB)
is larger than L2, so no flush is needed between steps.

--impl reference times the CPU oracle (plain FP64 C, OpenMP) on the host cores on a bounded
sample of the same workload, in the same metric.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("DOF-updates/s per RK stage (mixed Euler/NS-LES vs all-NS; FP32-TC vs FP64) at stated error")
UNIT = "DOF-updates/s"
THROTTLE_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
                 0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
                 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed_64x64x64_n4")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "tf32x3", "tf32"],
                    help="fp32: FP32 arithmetic with FP64 state and FP64 accumulation of q (the large "
                         "mixed configuration's precision); fp64: FP64 throughout")
    ap.add_argument("--no-extras", action="store_true", help="skip comparison, e2e and CPU baseline")
    ap.add_argument("--n", type=int, default=None, help="elements per direction (smaller profiling case)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--nodes", type=int, default=None, choices=[0, 1],
                    help="element nodes: 0 Gauss-Lobatto, 1 Gauss-Legendre (default: the workload's)")
    ap.add_argument("--tune-cache", default=None, help="autotuner cache file (read, then rewritten)")
    return ap.parse_args()


# ---- clocks --------------------------------------------------------------------------------

class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
               "--format=csv,noheader,nounits", "-lms", "10"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # nvidia-smi needs a moment before its first sample: wait for it (at most 3 s), so that
        # the samples cover the whole timed region that follows
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 4:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[3], 16)
            except ValueError:
                continue
            for b, name in THROTTLE_BITS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---- distributed -----------------------------------------------------------------------------

def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    # NCCL reduces device tensors; a CPU process group (gloo) host ones
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- CPU oracle baseline ---------------------------------------------------------------------

# DRAM traffic of the dominant kernel, from an ncu capture of this workload (committed under
# profiles/ with the hash of the kernel sources it was taken on); None once the sources differ.
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "traffic_stage_queue_fp32_mixed_64x64x64_n4.md")
# the same kernel's launches inside a chained call (every stage writes the next stage's traces)
TRAFFIC_RECORD_CHAINED = os.path.join(ROOT, "profiles", "traffic_stage_queue_chained_fp32_mixed_64x64x64_n4.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2403_05463_gb300", "csrc", f)
                  for f in ("dg_kernels_f32.cu", "dg_device.cuh", "dg_internal.h")]


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, the vendor's figure (context beside the measured peak)


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for path in KERNEL_SOURCES:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def stage_choice(tuning):
    """The autotuner's choice for an RK stage of one bucket: "separate" launches, one
    "persistent" kernel with a grid barrier, or one launch with "tile_queues"."""
    for line in tuning.splitlines():
        if line.startswith("stage "):
            head = line.split(" ms")[0]
            if "tile queues" in head:
                return "tile_queues"
            return "persistent" if "persistent kernel" in head else "separate"
    return "separate"


LAUNCH_NAMES = {"separate": "k_inviscid32t (the viscous pass a separate launch)",
                "persistent": "k_stage32t: viscous + inviscid + RK update, one cooperative launch per stage",
                "tile_queues": "k_stage32q: viscous + inviscid + RK update, one launch per stage (tile queues)"}


def recorded_traffic(workload, precision, n, kernel, launch, record=TRAFFIC_RECORD):
    """DRAM bytes per launch recorded for the one-launch stage kernel with tile queues on the
    benchmark workload, while the kernel sources hash to the recorded value."""
    if workload != "mixed_64x64x64_n4" or precision != "fp32" or n is not None or kernel != "inviscid_update" \
            or launch != "tile_queues":
        return None
    try:
        text = open(record).read()
    except OSError:
        return None
    import re
    m_t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    m_h = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", text)
    if not m_t or not m_h or m_h.group(1) != kernel_sources_sha256():
        return None
    return float(m_t.group(1))


def oracle_mesh(w, params=None):
    from oracle import oracle as orc
    m = w.mesh
    return orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, orc.params(**(params or w.params)), m.bc_tag)


def sampled_error(M, w, q_host, R_host, k=96, seed=7):
    """Relative L2 error of a residual computed by the library (host copy) against the FP64
    oracle, over the nodes of k randomly chosen elements (the oracle evaluates only those, with
    their neighbours' gradients): ||R - R_oracle|| / ||R_oracle|| and per variable (each
    variable's error over the same total norm)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(w.n_elem, min(k, w.n_elem), replace=False))
    R_ref = np.zeros_like(q_host)
    M.residual(q_host, sel=sel, out=R_ref)
    off = M.offsets
    idx = np.concatenate([np.arange(off[e], off[e + 1]) for e in sel])
    a, b = R_host[:, idx], R_ref[:, idx]
    nrm = float(np.sqrt((b ** 2).sum()))
    return {"rel_l2": float(np.sqrt(((a - b) ** 2).sum())) / nrm,
            "per_var": [float(np.sqrt(((a[v] - b[v]) ** 2).sum())) / nrm for v in range(a.shape[0])],
            "sample": f"{sel.size} random elements ({idx.size} nodes), FP64 oracle"}


def timed_steps(S, q, g, dt, stream, steps, warmup=2):
    """Mean milliseconds per RK3 step (CUDA events on the launching stream)."""
    import torch
    S.rk_step(q, g, dt, warmup, stream=stream)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    S.rk_step(q, g, dt, steps, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    S.check_device()
    return a.elapsed_time(b) / steps


def time_configs(S, w, q0, M, stream, hbm, device=0):
    """The metric's other points, outside the timed region: the same 64^3 mesh in FP64 and with
    the 3xTF32 tensor-core contraction; the precision-variant configuration (tgv 32^3, N = 5,
    30% NS slab) in FP32 and 3xTF32; the p-adaptive configuration (curved 32^3, orders 2..7,
    18.75% NS, one graph-captured step over every order bucket, autotuned). Each with its
    DOF-updates/s per stage and its residual error against the FP64 oracle on a sample."""
    import torch
    from paper_2403_05463_gb300 import dg, workloads as wl
    out = {}
    qh = q0.cpu().numpy()
    dof = S.total_nodes
    q = q0.clone()
    g = torch.zeros_like(q)
    div64 = {"fp64_divergence": 1}
    for prec, extra, steps in (("fp64", {}, 3), ("fp32", div64, 10), ("tf32x3", {}, 10), ("tf32x3", div64, 10)):
        S.set_params(dict(w.params, **extra), precision=prec)
        R = S.residual(q0).cpu().numpy()
        q.copy_(q0)
        ms = timed_steps(S, q, g, w.dt, stream, steps)
        key = f"{w.name}_{prec}" + ("_div64" if extra else "")
        out[key] = {"ms_per_step": ms, "value": dof * 3 / (ms * 1e-3), "dtype": prec,
                    "fp64_divergence": bool(extra), "error_vs_oracle": sampled_error(M, w, qh, R)}
        if prec == "fp64" or (prec == "fp32" and extra):
            # the mixed-vs-all-NS bar in the FP64 path and in the FP32 mode within 1e-6 of the oracle
            try:
                out[key]["comparison"] = cmp = flag_comparison(S, w, q0, q, g, stream, steps=steps,
                                                               reps=3 if prec == "fp32" else 1)
                if prec == "fp32":
                    # "at equal accuracy": the all-NS residual of this mode against the oracle too
                    import numpy as np
                    from oracle import oracle as orc
                    m = w.mesh
                    ones = np.ones(w.n_elem, np.uint8)
                    Mns = orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, ones, orc.params(**w.params), m.bc_tag)
                    S.set_flags(ones)
                    Rns = S.residual(q0).cpu().numpy()
                    S.set_flags(w.flags)
                    cmp["error_vs_oracle_mixed"] = out[key]["error_vs_oracle"]["rel_l2"]
                    cmp["error_vs_oracle_all_ns"] = sampled_error(Mns, w, qh, Rns)["rel_l2"]
                    del Mns, Rns
            except Exception as exc:  # an extra measurement must not cost the headline line
                S.set_flags(w.flags)
                out[key]["comparison"] = {"error": str(exc)}
    S.set_params(dict(w.params), precision="fp32")
    del q, g
    for name, make, variants in (("tgv_32x32x32_n5", wl.tgv_32x32x32_n5,
                                  (("fp32", {}), ("fp32", div64), ("tf32x3", {}), ("tf32x3", div64))),
                                 ("padapt_32x32x32", wl.padapt_32x32x32, (("fp32", {}),))):
        wc = make()
        Mc = oracle_mesh(wc)
        qc_h = wc.state(Mc.node_coords())
        for prec, extra in variants:
            Sc = dg.Solver.from_workload(wc, precision=prec, device=device, params=dict(wc.params, **extra))
            tuning = Sc.autotune() if prec == "fp32" else "default"
            qc = torch.from_numpy(qc_h).to(f"cuda:{device}")
            R = Sc.residual(qc).cpu().numpy()
            g = torch.zeros_like(qc)
            ms = timed_steps(Sc, qc, g, wc.dt, stream, 20)
            qc.copy_(torch.from_numpy(qc_h))
            ph_ms = Sc.phase_times(qc, g, wc.dt, reps=6, stream=stream)
            ph_b = Sc.phase_bytes()
            step_gb = 3 * sum(ph_b.values()) / 1e9
            out[f"{name}_{prec}" + ("_div64" if extra else "")] = {
                "ms_per_step": ms, "value": Sc.total_nodes * 3 / (ms * 1e-3), "dtype": prec,
                "fp64_divergence": bool(extra), "dof": Sc.total_nodes, "ns_fraction": wc.ns_fraction,
                "orders": sorted(int(o) for o in set(wc.orders.tolist())),
                "hbm_frac_step": step_gb / (ms * 1e-3) / hbm,
                "phases_ms": {k: v for k, v in ph_ms.items() if v > 0},
                "inviscid_update_gbs": ph_b["inviscid_update"] / (ph_ms["inviscid_update"] * 1e-3) / 1e9,
                "launches_per_step": Sc.launches_per_step, "launch_shapes": "autotuned" if tuning != "default" else tuning,
                "error_vs_oracle": sampled_error(Mc, wc, qc_h, R, k=128)}
            Sc.close()
            del qc, g
    return out


def timed_region_roofline(ph_ms, ph_bytes, ms_step, steps, hbm):
    """The one-launch stage kernel as it runs in the timed call of `steps` chained RK steps: one
    trace-kernel launch, then 3 * steps stage launches. In a chained call every stage's update
    writes the next stage's traces, so a launch moves the per-stage bytes of the viscous and
    inviscid passes (whose model has two of three stages writing traces) plus a third of one
    trace write (the trace phase's per-stage bytes are a third of a read and a write of the same
    size: half of them). Its mean duration is the timed region less the trace kernel's launch
    (timed on its own), over the stage launches."""
    launches = 3 * steps
    ms_launch = (ms_step * steps - ph_ms["traces"]) / launches
    nbytes = ph_bytes["inviscid_update"] + 0.5 * ph_bytes["traces"]
    ach = nbytes / (ms_launch * 1e-3) / 1e9
    return {"achieved": ach, "frac": ach / hbm, "bytes_per_launch": nbytes, "ms_per_launch": ms_launch,
            "launches": launches}


def flag_comparison(S, w, q0, q, g, stream, steps, reps):
    """Chained steps with the workload's flags, all NS and all Euler on the same mesh and GPU
    (each set timed reps times, interleaved; the median of each) and the bar
    T_mixed <= f T_allNS + (1 - f) T_allEuler."""
    import numpy as np
    runs = {"mixed": [], "all_ns": [], "all_euler": []}
    sets = (("mixed", w.flags), ("all_ns", np.ones(w.n_elem, np.uint8)), ("all_euler", np.zeros(w.n_elem, np.uint8)))
    for _ in range(reps):
        for name, fl in sets:
            S.set_flags(fl)
            q.copy_(q0)
            runs[name].append(timed_steps(S, q, g, w.dt, stream, steps, warmup=2))
    S.set_flags(w.flags)
    med = {k: statistics.median(v) for k, v in runs.items()}
    f = w.ns_fraction
    bar = f * med["all_ns"] + (1 - f) * med["all_euler"]
    return {"mixed_ms_per_step": med["mixed"], "all_ns_ms_per_step": med["all_ns"],
            "all_euler_ms_per_step": med["all_euler"], "bar_ms_per_step": bar, "meets_bar": med["mixed"] <= bar,
            "speedup_vs_all_ns": med["all_ns"] / med["mixed"], "steps": steps, "runs": reps}


def oracle_rate(w, q_host, budget_s=20.0, seed=0, M=None):
    """The FP64 oracle as it stands, on the host cores: residual of a random sample of
    elements (each needs its neighbours' BR1 gradients too), DOF of the sample / wall time."""
    import numpy as np
    from oracle import oracle as orc
    if M is None:
        M = oracle_mesh(w)
    rng = np.random.default_rng(seed)
    n3 = (w.orders.astype(np.int64) + 1) ** 3
    R = np.zeros_like(q_host)

    def timed(k):
        sel = np.sort(rng.choice(w.n_elem, size=min(k, w.n_elem), replace=False))
        t0 = time.perf_counter()
        M.residual(q_host, sel=sel, out=R)
        return float(n3[sel].sum()), time.perf_counter() - t0, sel.size

    dof, dt, _ = timed(256)
    k = int(min(w.n_elem, max(256, 256 * budget_s / max(dt, 1e-3))))
    dof, dt, k = timed(k)
    cores = orc.num_threads()
    out = {"value": dof / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"one FP64 residual of {k} randomly sampled elements of {w.name} "
                     f"({int(dof)} DOF, {dt:.1f} s; neighbours' gradients included in the time)"}
    # and on one core, a smaller sample
    orc.set_num_threads(1)
    try:
        dof1, dt1, k1 = timed(max(16, int(k * 3.0 / budget_s / max(cores, 1))))
    finally:
        orc.set_num_threads(cores)
    out["one_core"] = {"value": dof1 / dt1, "sample": f"{k1} elements, {int(dof1)} DOF, {dt1:.1f} s"}
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as orc
    from paper_2403_05463_gb300 import workloads as wl
    w = wl.WORKLOADS[args.workload]()
    m = w.mesh
    M = orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, orc.params(**w.params), m.bc_tag)
    xyz = M.node_coords()
    q = w.state(xyz)
    del xyz
    n3 = (w.orders.astype(np.int64) + 1) ** 3
    rng = np.random.default_rng(1)
    R = np.zeros_like(q)
    # size one step (one stage on a sample) so that warmup + steps fit in about two minutes
    sel = rng.choice(w.n_elem, 128, replace=False)
    t0 = time.perf_counter()
    M.residual(q, sel=sel, out=R)
    per_elem = (time.perf_counter() - t0) / sel.size
    k = int(max(64, min(w.n_elem, 100.0 / max(1, args.steps + args.warmup) / max(per_elem, 1e-6))))
    times, dofs = [], []
    for i in range(args.warmup + args.steps):
        sel = np.sort(rng.choice(w.n_elem, k, replace=False))
        t0 = time.perf_counter()
        M.residual(q, sel=sel, out=R)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            dofs.append(float(n3[sel].sum()))
    value = sum(dofs) / sum(times)
    ms = 1e3 * sum(times) / len(times)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": w.name, "n_elem": int(w.n_elem), "dof": int(w.total_nodes),
                      "ns_fraction": w.ns_fraction, "step": f"one residual (one RK stage) of {k} sampled elements"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                            "sample": f"{k} randomly sampled elements per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ---- GPU -------------------------------------------------------------------------------------

# A fixed two-component mixture in the feature units of the synthetic turbulence of the 64^3
# workload (there Q_S ~ -0.23, Q_Omega ~ 0.21 at the median): a narrow low-gradient component
# and a broad strongly rotational one; it flags about a third of the elements. The detection
# pass costs the same whatever the mixture.
BENCH_GMM = {"weights": [0.7, 0.3], "means": [[-0.15, 0.0, 0.1], [-0.45, 0.0, 0.45]],
             "covs": [[[0.01, 0, 0], [0, 1e-4, 0], [0, 0, 0.01]], [[0.1, 0, 0], [0, 1e-3, 0], [0, 0, 0.12]]],
             "viscous": 1}


def time_detection(S, w, q, q0, stream, reps=10):
    """Mean time of dg_detect_regions (flags and element means, no node features), FP64 and
    FP32 passes, with CUDA events on the launching stream, and the algorithmic bytes: the three
    velocity planes, the metric terms (per element on box/affine meshes, per node on curved
    ones) and the outputs; the two passes' flags are compared."""
    import torch
    q.copy_(q0)
    total, ne = S.total_nodes, S.n_elem
    curved = w.mesh.geom_degree > 1
    out, flags = {}, {}
    for prec, name in ((0, "fp64"), (1, "fp32")):
        for _ in range(3):
            S.detect_regions(q, BENCH_GMM, precision=prec, stream=stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fl, pb, _ = S.detect_regions(q, BENCH_GMM, precision=prec, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        geo_bytes = (40 if prec else 80) * (total if curved else 1) * (1 if curved else ne)
        nbytes = 24 * total + geo_bytes + 17 * ne
        flags[name] = fl
        out[name] = {"ms": ms, "algorithmic_gb": nbytes / 1e9, "gbs": nbytes / (ms * 1e-3) / 1e9,
                     "viscous_fraction": float(fl.double().mean()), "node_rate": total / (ms * 1e-3)}
    out["flags_agree"] = float((flags["fp64"] == flags["fp32"]).double().mean())
    return out


def time_compressible(stream, device=0, steps=10):
    """RK3 steps of the compressible form (FP64) on cns_tgv 32^3 N = 4 (4.1 M nodes, 30% NS;
    u + g = 0.33 GB, above L2): CUDA events on the launching stream, per-phase times and the
    algorithmic bytes of each phase; then the same steps on Gauss-Legendre nodes."""
    import numpy as np
    import torch
    from paper_2403_05463_gb300 import dg, workloads as wl
    w = wl.cns_tgv(n=32, order=4)
    S = dg.Solver.from_workload(w, precision=0, device=device)
    xyz = S.node_coords()
    u = torch.from_numpy(wl.cns_state(xyz.cpu().numpy(), w.seed, period=2 * np.pi)).to(xyz.device)
    g = torch.zeros_like(u)
    for _ in range(3):
        S.rk_step(u, g, w.dt, 1, stream=stream)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    S.rk_step(u, g, w.dt, steps, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    ph_ms = S.phase_times(u, g, w.dt, reps=3, stream=stream)
    ph_b = S.phase_bytes()
    S.check_device()
    dof = S.total_nodes
    del S, u, g
    Sg = dg.Solver.from_workload(w, precision=0, device=device, params=dict(w.params, nodes=1))
    xg = Sg.node_coords()
    u = torch.from_numpy(wl.cns_state(xg.cpu().numpy(), w.seed, period=2 * np.pi)).to(xg.device)
    g = torch.zeros_like(u)
    for _ in range(3):
        Sg.rk_step(u, g, w.dt, 1, stream=stream)
    a.record(stream)
    Sg.rk_step(u, g, w.dt, steps, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms_gl = a.elapsed_time(b) / steps
    Sg.check_device()
    return {"workload": w.name, "dtype": "f64", "ms_per_step": ms, "value": dof * 3 / (ms * 1e-3),
            "unit": UNIT, "ns_fraction": w.ns_fraction,
            "phases": {k: {"ms": ph_ms[k], "algorithmic_gb": ph_b[k] / 1e9} for k in ph_ms if ph_ms[k] > 0},
            "gauss_legendre": {"ms_per_step": ms_gl, "value": dof * 3 / (ms_gl * 1e-3)}}


def time_gauss_legendre(stream, device=0, steps=5):
    """FP64 RK3 steps of the incompressible form on tgv 32^3 N = 5 (4.4 M nodes, 30% NS) on
    Gauss-Lobatto and on Gauss-Legendre element nodes, CUDA events on the launching stream."""
    import torch
    from paper_2403_05463_gb300 import dg, workloads as wl
    w = wl.tgv_32x32x32_n5()
    out = {"workload": w.name, "dtype": "f64", "unit": UNIT}
    for nodes, name in ((0, "gauss_lobatto"), (1, "gauss_legendre")):
        S = dg.Solver.from_workload(w, precision=0, device=device, params=dict(w.params, nodes=nodes))
        xyz = S.node_coords()
        q = torch.from_numpy(w.state(xyz.cpu().numpy())).to(xyz.device)
        g = torch.zeros_like(q)
        S.rk_step(q, g, w.dt, 2, stream=stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        S.rk_step(q, g, w.dt, steps, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        S.check_device()
        ms = a.elapsed_time(b) / steps
        out[name] = {"ms_per_step": ms, "value": S.total_nodes * 3 / (ms * 1e-3)}
        del S, q, g, xyz
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    from paper_2403_05463_gb300 import dg, workloads as wl

    world, rank, local = dist_setup()
    w = wl.WORKLOADS[args.workload]() if args.n is None else wl.WORKLOADS[args.workload](n=args.n)
    if args.nodes is not None:
        w = dataclasses.replace(w, params=dict(w.params, nodes=args.nodes))
    S = dg.Solver.from_workload(w, precision=args.precision, device=local)
    # launch shapes per (order, geometry) timed on this GPU and mesh before the timed region
    tuning = "default" if args.no_autotune else S.autotune(args.tune_cache)
    dof = S.total_nodes
    xyz = S.node_coords()
    q = w.state_fn(xyz, None, None) if args.workload == "mixed_64x64x64_n4" else \
        torch.from_numpy(w.state(xyz.cpu().numpy())).cuda()
    q = q.contiguous()
    del xyz
    q0 = q.clone()
    g = torch.zeros_like(q)
    dt = w.dt
    stream = torch.cuda.current_stream()

    # K steps are one dg_rk_step call: the steps are chained (every stage's update writes the
    # next stage's traces, so only the first step runs the trace kernel)
    if args.warmup > 0:
        S.rk_step(q, g, dt, args.warmup, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()  # returns once the sampler has its first sample
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    S.rk_step(q, g, dt, args.steps, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = allmax(world, ms)
    value = world * dof * 3 / (ms_max * 1e-3)
    S.check_device()
    launches = S.launches_per_step + S.launches_per_chained_step * (args.steps - 1) if args.steps > 1 else \
        S.launches_per_step * args.steps

    # roofline of the dominant phase (CUDA events between the phases, same stream)
    q.copy_(q0)
    ph_ms = S.phase_times(q, g, dt, reps=6, stream=stream)
    ph_bytes = S.phase_bytes()
    dom = max(ph_ms, key=lambda k: ph_ms[k])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ach = ph_bytes[dom] / (ph_ms[dom] * 1e-3) / 1e9
    # the timed call's bytes per step: every step's three stages, the trace kernel in the first
    # step only, and in every step a third update writing traces (ph_bytes are per-stage means:
    # the trace kernel's launch moves 3 x traces, half of it the written traces)
    step_bytes = 3 * sum(ph_bytes.values()) - (1.5 * ph_bytes["traces"] * (args.steps - 1) / max(args.steps, 1))
    launch = stage_choice(tuning) if tuning != "default" else "separate"
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "launch": LAUNCH_NAMES[launch] if dom == "inviscid_update" else dom,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "nominal_peak": NOMINAL_HBM_GBS, "frac_nominal": ach / NOMINAL_HBM_GBS,
                "traffic": recorded_traffic(args.workload, args.precision, args.n, dom, launch),
                "step_frac": step_bytes / (ms_max * 1e-3) / 1e9 / hbm}
    if launch in ("tile_queues", "persistent") and dom == "inviscid_update" and args.steps > 1 \
            and ph_ms.get("traces", 0.0) > 0.0:
        # the dominant kernel as it runs in the timed region (chained launches); the launches
        # timed on their own (plain stages, stage 2 writing no traces) stay beside it
        try:
            tr = timed_region_roofline(ph_ms, ph_bytes, ms_max, args.steps, hbm)
            roofline["isolated"] = {"achieved": ach, "frac": ach / hbm, "traffic": roofline["traffic"],
                                    "how": "phase timing: plain stage launches, per-stage mean bytes"}
            roofline.update({"achieved": tr["achieved"], "frac": tr["frac"],
                             "frac_nominal": tr["achieved"] / NOMINAL_HBM_GBS,
                             "traffic": recorded_traffic(args.workload, args.precision, args.n, dom, launch,
                                                         TRAFFIC_RECORD_CHAINED),
                             "how": f"timed region: {tr['launches']} chained stage launches, "
                                    f"{tr['bytes_per_launch'] / 1e9:.3f} GB and {tr['ms_per_launch']:.4f} ms "
                                    "per launch (the trace kernel's launch taken out)"})
        except Exception as exc:  # keep the isolated figure
            roofline["timed_region_error"] = str(exc)
    phases = {k: {"ms": ph_ms[k], "algorithmic_gb": ph_bytes[k] / 1e9,
                  "gbs": (ph_bytes[k] / (ph_ms[k] * 1e-3) / 1e9) if ph_ms[k] > 0 else None} for k in ph_ms}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "tf32x3": "tf32x3", "tf32": "tf32"}[args.precision], "data": "synthetic",
           "config": {"workload": w.name, "n_elem": int(w.n_elem), "order": int(w.orders.max()), "dof": int(dof),
                      "ns_fraction": w.ns_fraction, "precision": args.precision, "stages_per_step": 3,
                      "state": "FP64 q, g resident in HBM; FP64 RK accumulation",
                      "l2": f"inputs larger than L2 (q + g = {2 * q.numel() * 8 / 1e9:.2f} GB per rank)",
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "launch_shapes": "default" if tuning == "default" else "autotuned: " +
                      "; ".join(line.split(" ms")[0].split(":")[0] + ":" + line.split(":")[1]
                                for line in tuning.strip().splitlines() if ":" in line)},
           "roofline": roofline, "phases": phases, "gpu_launches": launches, "clocks": clk}
    # the autotuner's stage choice: one persistent kernel per RK stage (viscous pass, grid
    # barrier, inviscid pass) against separate launches, both timed on its scratch state
    for line in tuning.splitlines():
        if line.startswith("stage ") and "persistent kernel" in line and "separate" in line:
            import re
            m = re.search(r"one persistent kernel ([0-9.]+) ms, one launch with tile queues ([0-9.]+) ms, "
                          r"separate ([0-9.]+) ms", line)
            if m:
                out["stage_kernel"] = {"chosen": stage_choice(line), "persistent_ms_per_stage": float(m.group(1)),
                                       "tile_queues_ms_per_stage": float(m.group(2)),
                                       "separate_ms_per_stage": float(m.group(3))}
                ms = re.search(r"blocks starting with the viscous tiles: ([^)]*)\)", line)
                if ms:
                    out["stage_kernel"]["queue_viscous_first_blocks"] = ms.group(1)

    if not args.no_extras:
        # mixed vs all-NS and all-Euler on the same mesh and GPU
        # each flag set timed three times, interleaved (20 chained steps after 3 warm-up steps):
        # the median of the three
        cmp = {}
        bytes_mixed = 3 * sum(S.phase_bytes().values())
        runs = {"mixed": [], "all_ns": [], "all_euler": []}
        sets = (("mixed", w.flags), ("all_ns", np.ones(w.n_elem, np.uint8)), ("all_euler", np.zeros(w.n_elem, np.uint8)))
        for _ in range(3):
            for name, fl in sets:
                S.set_flags(fl)
                if name == "all_ns":
                    bytes_ns = 3 * sum(S.phase_bytes().values())
                q.copy_(q0)
                runs[name].append(timed_steps(S, q, g, dt, stream, 20, warmup=3))
        S.set_flags(w.flags)
        for name in ("all_ns", "all_euler"):
            t = statistics.median(runs[name])
            cmp[name] = {"ms_per_step": t, "value": dof * 3 / (t * 1e-3), "runs_ms": runs[name]}
        ms_mixed = statistics.median(runs["mixed"])
        # "at equal accuracy": what dropping the viscous terms in the Euler elements changes,
        # the residual of the flagged run against the all-NS one on the Euler elements
        q.copy_(q0)
        R_mixed = S.residual(q)
        S.set_flags(np.ones(w.n_elem, np.uint8))
        R_ns = S.residual(q)
        S.set_flags(w.flags)
        n_el = np.diff(S.offsets)
        euler_nodes = torch.from_numpy(np.repeat(w.flags == 0, n_el)).to(q.device)
        dR = (R_mixed - R_ns)[:, euler_nodes]
        cmp["euler_elements_rel_residual_change"] = float(torch.linalg.norm(dR) /
                                                          torch.linalg.norm(R_ns[:, euler_nodes]))
        del R_mixed, R_ns, dR, euler_nodes
        f = w.ns_fraction
        bar = f * cmp["all_ns"]["ms_per_step"] + (1 - f) * cmp["all_euler"]["ms_per_step"]
        cmp["mixed_ms_per_step"] = ms_mixed
        cmp["mixed_runs_ms"] = runs["mixed"]
        cmp["bar_ms_per_step"] = bar
        cmp["speedup_vs_all_ns"] = cmp["all_ns"]["ms_per_step"] / ms_mixed
        cmp["meets_bar"] = ms_mixed <= bar
        # the same bar in the byte model's form: the speedup over all-NS that the algorithmic
        # bytes predict, W_allNS / W_mixed
        cmp["byte_model_speedup"] = bytes_ns / bytes_mixed
        cmp["meets_byte_model_bar"] = cmp["speedup_vs_all_ns"] >= cmp["byte_model_speedup"]
        out["comparison"] = cmp
        # overlapped launches (the default) against plain ones, same mesh and flags: 20 chained
        # steps each, alternated twice
        ov = {"on": [], "off": []}
        for _ in range(2):
            for name, on in (("off", False), ("on", True)):
                S.set_launch_overlap(on)
                q.copy_(q0)
                ov[name].append(timed_steps(S, q, g, dt, stream, 20, warmup=3))
        S.set_launch_overlap(True)
        out["launch_overlap"] = {"on_ms_per_step": sum(ov["on"]) / 2, "off_ms_per_step": sum(ov["off"]) / 2,
                                 "steps": 20}
        # region detection (Sec. 2.1) on the benchmark state: one pass over the whole mesh
        out["detect"] = time_detection(S, w, q, q0, stream)
        # the compressible form (App. A), FP64, on its own periodic workload
        out["compressible"] = time_compressible(stream, device=local)
        # Gauss-Legendre element nodes (App. B's quadrature) against Gauss-Lobatto, FP64
        out["gauss_legendre"] = time_gauss_legendre(stream, device=local)
        # end to end through the C ABI with host buffers (pinned), copies inside the timing:
        # every step copies the state in and the new state out (the RK register, which the
        # first stage overwrites unread, stays on the device)
        qh = q0.cpu().pin_memory()
        S.rk_step_host(qh, None, dt, 1, stream=stream)
        n_e2e = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            S.rk_step_host(qh, None, dt, 1, stream=stream)
        t_e2e = (time.perf_counter() - t0) / n_e2e
        t_e2e = allmax(world, t_e2e)
        nbytes = qh.numel() * 8
        out["e2e"] = {"value": world * dof * 3 / t_e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": nbytes, "ms_per_step": t_e2e * 1e3}
        if rank == 0 and world == 1:
            M = oracle_mesh(w)
            qh0 = q0.cpu().numpy()
            # the headline's accuracy: the benchmarked residual against the FP64 oracle
            out["error_vs_oracle"] = err = sampled_error(M, w, qh0, S.residual(q0).cpu().numpy())
            if args.precision != "fp64":
                # which row carries the error, and the configuration that removes it
                names = ("p", "u", "v", "w")
                worst = max(range(4), key=lambda v: err["per_var"][v])
                err["dominant_variable"] = names[worst]
                if worst == 0:
                    err["cause"] = ("pressure row: R_p = -c0^2 div u of a nearly divergence-free field is a "
                                    "small difference of three FP32 directional derivatives; the FP64 "
                                    "velocity divergence (configs: *_div64) removes it")
            out["configs"] = time_configs(S, w, q0, M, stream, hbm, device=local)
            try:
                out["cpu_baseline"] = oracle_rate(w, qh0, M=M)
            except Exception as exc:  # the baseline is context, never the product path
                out["cpu_baseline"] = {"value": None, "unit": UNIT, "kind": "oracle", "cores": None,
                                       "sample": f"not measured: {exc}"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
