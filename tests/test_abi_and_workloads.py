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


class _FakeTensor:
    """Stands in for a CUDA tensor of the wrong size: the size checks must refuse it before any
    pointer is taken or any library call is made."""
    def __init__(self, n):
        self._n = n

    def numel(self):
        return self._n


def _sized_solver(monkeypatch, total=100, before=None):
    class Sized(dg.Solver):
        total_nodes = total  # no library call

    S = Sized.__new__(Sized)
    S.params, S.h, S.n_elem = {}, None, 1
    if before is not None:
        S._total_before_orders = before

    def no_library():
        raise AssertionError("the library was called")
    monkeypatch.setattr(dg, "load", no_library)
    return S


def test_noalloc_sums_refuse_a_wrongly_sized_R_without_a_launch(monkeypatch):
    S = _sized_solver(monkeypatch)
    with pytest.raises(ValueError, match=r"R must hold \[4\]\[100\]"):
        S.conservation_noalloc(_FakeTensor(4 * 99), _FakeTensor(4))


def test_project_state_refuses_a_q_old_of_another_layout(monkeypatch):
    pytest.importorskip("torch")
    S = _sized_solver(monkeypatch, total=100, before=64)
    with pytest.raises(ValueError, match=r"q_old must hold \[4\]\[64\]"):
        S.project_state(_FakeTensor(4 * 100))
    S5 = _sized_solver(monkeypatch, total=100, before=64)
    S5.params = {"model": 1}
    with pytest.raises(ValueError, match=r"q_old must hold \[5\]\[64\]"):
        S5.project_state(_FakeTensor(4 * 64))  # a four-plane state for the five-plane form


def test_product_path_shares_nothing_with_the_oracle():
    # the library, its binding and its headers neither import, include, link nor load anything
    # under oracle/, and the oracle includes nothing of the library
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pat = re.compile(r"(import\s+oracle|from\s+oracle|liboracle|dg_oracle|oracle/)")
    product = [os.path.join(root, "include")] + [os.path.join(root, "paper_2403_05463_gb300")]
    for top in product:
        for dirpath, _, files in os.walk(top):
            if "_build" in dirpath or "__pycache__" in dirpath:
                continue
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                    text = open(os.path.join(dirpath, f), encoding="utf-8").read()
                    assert not pat.search(text), os.path.join(dirpath, f)
    inc = re.compile(r'#include\s+"([^"]+)"')
    for f in os.listdir(os.path.join(root, "oracle")):
        if f.endswith((".c", ".h")):
            text = open(os.path.join(root, "oracle", f), encoding="utf-8").read()
            assert all(h.startswith("dg_oracle") for h in inc.findall(text)), f
