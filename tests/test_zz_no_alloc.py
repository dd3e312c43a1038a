"""dg_conservation_noalloc, the conservation sums for callers that cannot allocate device memory
while they run, through the C ABI.

Its output is checked against two things on the same R: dg_conservation (the library's
allocating call, host-side final sum) and the oracle's weighted sums, which take their own
quadrature weights and Jacobians, so a mistake in the weights or in J common to both library
calls still fails. The device's free memory must not change across repeated calls. Collected
last, so it runs both after the other GPU tests and, alone, in a fresh process (the first call on
the device does the scratch look-up)."""
import numpy as np
import pytest

from paper_2403_05463_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity tolerance (relative)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _solver(w, precision=0, params=None):
    from paper_2403_05463_gb300 import dg
    return dg.Solver.from_workload(w, precision=precision, params=params)


def _oracle(w, params=None):
    from oracle import oracle as orc
    m = w.mesh
    return orc.Mesh(m.hex, m.geom, m.geom_degree, w.orders, w.flags, orc.params(**(params or w.params)), m.bc_tag)


def _random_R(S, seed):
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    # positive mean: the weighted sums are far from zero, so a relative bound is meaningful
    return (0.5 + torch.rand((4, S.total_nodes), generator=g, dtype=torch.float64)).cuda()


def _check_two_calls(S, M=None):
    import torch
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    for seed in (1, 2):  # two calls in a row, different inputs, same shared scratch
        R = _random_R(S, seed)
        S.conservation_noalloc(R, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = S.conservation(R)
        assert np.all(np.isfinite(got)), got
        assert np.all(np.abs(got - ref) <= TOL * np.abs(ref)), (seed, got, ref)
        if M is not None:
            ind = M.conservation(R.cpu().numpy())  # the oracle's weights and J
            assert np.all(np.abs(got - ind) <= TOL * np.abs(ind)), (seed, got, ind)


def test_noalloc_matches_conservation_curved_mixed_orders():
    # curved geometry (per-node J) and orders 2..7: several order buckets fill the scratch
    w = wl.padapt_32x32x32(n=6)
    _check_two_calls(_solver(w), _oracle(w))


def test_noalloc_matches_the_oracle_under_fp32_arithmetic():
    # the reduced-precision context keeps FP64 geometry for the sums: same result
    w = wl.padapt_32x32x32(n=6)
    _check_two_calls(_solver(w, precision=1), _oracle(w))


def test_noalloc_matches_the_oracle_on_gauss_points():
    w = wl.padapt_32x32x32(n=5)
    prm = dict(w.params, nodes=1)
    _check_two_calls(_solver(w, params=prm), _oracle(w, prm))


def test_noalloc_at_the_scratch_limit():
    n = 40  # 64000 elements, just under the 65536-element limit
    w = wl.tgv_4x4x4_n3(n_elem_dir=n, order=1)
    _check_two_calls(_solver(w), _oracle(w))


def test_noalloc_leaves_device_memory_unchanged():
    import torch
    w = wl.padapt_32x32x32(n=6)
    S = _solver(w)
    R = _random_R(S, 4)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    first = torch.zeros(4, dtype=torch.float64, device="cuda")
    S.conservation_noalloc(R, first)  # the first call loads the kernels and looks up the scratch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(20):
        S.conservation_noalloc(R, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_reserved() == reserved0
    assert torch.equal(out, first)  # fixed summation order: identical sums every call


def test_noalloc_rejects_a_mesh_beyond_the_limit():
    import torch
    from paper_2403_05463_gb300 import dg
    S = _solver(wl.tgv_4x4x4_n3(n_elem_dir=41, order=1))  # 68921 elements
    R = _random_R(S, 3)
    out = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as ei:
        S.conservation_noalloc(R, out)
    assert dg.STATUS[ei.value.status] == "DG_ERR_ARG" and "scratch holds" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)  # nothing was launched
