"""dg_conservation_noalloc (allocation-free conservation sums into caller-owned device memory)
against dg_conservation, through the C ABI. Collected last, so it runs both after the other
GPU tests and, alone, in a fresh process (the first call on the device does the scratch
look-up)."""
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


def _solver(w):
    from paper_2403_05463_gb300 import dg
    return dg.Solver.from_workload(w, precision=0)


def _random_R(S, seed):
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    # positive mean: the weighted sums are far from zero, so a relative bound is meaningful
    return (0.5 + torch.rand((4, S.total_nodes), generator=g, dtype=torch.float64)).cuda()


def _check_two_calls(S):
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


def test_noalloc_matches_conservation_curved_mixed_orders():
    # curved geometry (per-node J) and orders 2..7: several order buckets fill the scratch
    _check_two_calls(_solver(wl.padapt_32x32x32(n=6)))


def test_noalloc_at_the_scratch_limit():
    n = 40  # 64000 elements, just under the 65536-element limit
    _check_two_calls(_solver(wl.tgv_4x4x4_n3(n_elem_dir=n, order=1)))


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
