"""CPU tests: the C-ABI library builds, loads and exports every symbol include/dg.h declares;
the seeded workload generator produces the specified shapes (no GPU calls)."""
import ctypes

import numpy as np
import pytest

from paper_2403_05463_gb300 import dg, workloads as wl


@pytest.fixture(scope="module")
def lib():
    from paper_2403_05463_gb300 import build
    build.build()
    return ctypes.CDLL(dg.LIB_PATH)


def test_library_exports_every_declared_symbol(lib):
    names = dg.header_symbols()
    assert "dg_create_mesh" in names and "dg_rk_step" in names and "dg_residual" in names
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_loads_and_reports_errors_without_gpu(lib):
    L = dg.load()
    # a NULL descriptor is rejected before any CUDA call
    h = ctypes.c_void_p()
    st = L.dg_create_mesh(None, None, 0, ctypes.byref(h))
    assert st == 1 and not h.value
    assert b"NULL" in L.dg_last_error()
    assert L.dg_launches_per_step(None) == 0
    L.dg_destroy(None)


def test_workload_shapes():
    w = wl.wake_16x16x16_n4()
    assert w.n_elem == 4096 and w.total_nodes == 512000
    assert int(w.flags.sum()) == 512  # 32 of 256 cross-section columns
    assert (w.mesh.bc_tag == 1).sum() == 256 and (w.mesh.bc_tag == 2).sum() == 256
    w3 = wl.tgv_32x32x32_n5()
    assert int(w3.flags.sum()) == round(0.3 * 32768)
    f = w3.flags
    assert np.count_nonzero(np.diff(np.r_[f, f[:1]].astype(int)) != 0) == 2  # one contiguous run
    w5 = wl.mixed_64x64x64_n4()
    assert w5.total_nodes == 32768000
    assert 0.23 < w5.ns_fraction < 0.27
    w4 = wl.padapt_32x32x32()
    assert set(np.unique(w4.orders)) <= set(range(2, 8))
    core = np.abs(w4.mesh.centers[:, 1] - 0.5) < 0.1
    assert np.all(w4.flags[core] == 1) and np.all(w4.flags[~core] == 0)
    assert set(np.unique(w4.orders[core])) == {6, 7}


def test_noise_is_layout_independent():
    e = np.array([5, 7, 5])
    l = np.array([3, 3, 3])
    a = wl.node_noise(1003, e, l, 2, 0.01)
    assert a[0] == a[2] and a[0] != a[1]
    assert np.all(np.abs(wl.node_noise(1, np.arange(1000), np.zeros(1000, int), 0, 0.01)) <= 0.01)


def test_kraichnan_modes_are_divergence_free_and_scaled():
    m = wl.kraichnan_modes(1005, (8.0, 4.0, 4.0))
    assert np.abs((m.k * m.amp).sum(axis=1)).max() < 1e-12
    assert abs(np.sqrt((m.amp ** 2).sum() / 6.0) - 0.05) < 1e-12
    L = np.array([8.0, 4.0, 4.0])
    n = m.k * L / (2 * np.pi)
    assert np.abs(n - np.round(n)).max() < 1e-9  # periodic on the box


def test_bench_and_entry_compile():
    import py_compile
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for f in ("bench.py", "__graft_entry__.py"):
        py_compile.compile(os.path.join(root, f), doraise=True)
