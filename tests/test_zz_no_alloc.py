"""The allocation-free entry point (tb_amplitudes_noalloc) against the
workspace entry point (tb_amplitudes_device), through the C-ABI.

Callers that cannot allocate device memory when they need amplitudes (a
process whose device memory is capped by someone else's quota, a plugin whose
host application tracks every device allocation) use the library's fixed
scratch array instead of a workspace. Its results
must match the workspace path on consecutive calls, since every call reuses
whatever the previous one left in that array. This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def tb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13110_gb300 import build as b
    b.build()
    import paper_2608_13110_gb300 as mod
    return mod


@pytest.mark.parametrize("n,d", [(20, 36), (12, 8)])  # HBM-pass path (width 18) and narrow path
def test_noalloc_matches_workspace_entry_on_two_calls(tb, n, d):
    import torch
    c = W.random_circuit(n, d, None, 6, 500 + d)
    plan = tb.Plan.from_circuit(c)
    ws = plan.alloc_workspace(6)
    plan.upload(ws)
    d_bits = torch.from_numpy(c.bits).cuda()
    ref = torch.empty((6, 2), dtype=torch.float64, device="cuda")
    plan.amplitudes_device(d_bits, ws, ref)
    torch.cuda.synchronize()
    r = ref.cpu().numpy().view(np.complex128).reshape(-1)
    for _ in range(2):
        out = torch.full((6, 2), float("nan"), dtype=torch.float64, device="cuda")
        plan.amplitudes_noalloc(d_bits, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy().view(np.complex128).reshape(-1)
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) / np.linalg.norm(r) <= TOL


def test_noalloc_rejects_circuits_beyond_the_scratch(tb):
    import torch
    plan = tb.Plan(30, 48)  # width 24: a 128 MiB boundary does not fit 64 MiB
    d_bits = torch.zeros((1, 30), dtype=torch.uint8, device="cuda")
    out = torch.empty((1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(tb.TbError) as e:
        plan.amplitudes_noalloc(d_bits, out)
    assert e.value.status == tb.TB_ENOMEM
