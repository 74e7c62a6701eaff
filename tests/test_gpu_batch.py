"""Batches of uneven circuits recorded into one CUDA graph (tb_batch_*):
every amplitude equals the single-circuit entry point's, bit for bit, on
repeated launches, and narrow circuits match the FP64 state vector."""
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


def _single(tb, plan, bits):
    import torch
    nb = bits.shape[0]
    ws = plan.alloc_workspace(nb)
    plan.upload(ws)
    d_bits = torch.from_numpy(bits).cuda()
    out = torch.empty((nb, 2), dtype=torch.float64, device="cuda")
    plan.amplitudes_device(d_bits, ws, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.complex128).reshape(-1)


def _run_batch(tb, circuits, nbranches=0):
    import torch
    plans = [tb.Plan.from_circuit(c) for c in circuits]
    d_bits = [torch.from_numpy(c.bits).cuda() for c in circuits]
    d_out = [torch.full((c.bits.shape[0], 2), float("nan"), dtype=torch.float64, device="cuda")
             for c in circuits]
    batch = tb.Batch(list(zip(plans, d_bits, d_out)), nbranches=nbranches)
    return plans, d_out, batch


def test_mixed_batch_matches_single_calls_and_oracle(tb, oracle_mod):
    import torch
    shapes = [(12, 8, 16), (9, 20, 8), (14, 26, 6), (20, 34, 5), (18, 30, 7), (6, 16, 32), (11, 24, 3), (2, 28, 4)]
    circuits = [W.random_circuit(n, d, None, nb, 600 + i) for i, (n, d, nb) in enumerate(shapes)]
    plans, d_out, batch = _run_batch(tb, circuits, nbranches=3)
    for rep in range(2):
        for o in d_out:
            o.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        for c, plan, o in zip(circuits, plans, d_out):
            got = o.cpu().numpy().view(np.complex128).reshape(-1)
            np.testing.assert_array_equal(got, _single(tb, plan, c.bits))
            if c.n <= 14:
                ref = oracle_mod.sv_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), c.bits)
                assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL


def test_uneven_batch_shape_of_the_batching_workload(tb):
    """A scaled-down draw of the 64-circuit workload: n in [20, 70], d even in
    [16, 48] (widths 8..24), every circuit different."""
    import torch
    circuits = W.batch_uneven(n_circuits=10, nb=3)
    plans, d_out, batch = _run_batch(tb, circuits)
    batch.launch()
    torch.cuda.synchronize()
    for c, plan, o in zip(circuits, plans, d_out):
        got = o.cpu().numpy().view(np.complex128).reshape(-1)
        np.testing.assert_array_equal(got, _single(tb, plan, c.bits))


def test_batch_rejects_a_short_workspace(tb):
    import ctypes
    import torch
    c = W.random_circuit(16, 30, None, 2, 7)
    plan = tb.Plan.from_circuit(c)
    d_bits = torch.from_numpy(c.bits).cuda()
    d_out = torch.empty((2, 2), dtype=torch.float64, device="cuda")
    arr = (tb._BatchItem * 1)()
    arr[0].plan = plan.handle.value
    arr[0].d_bits = d_bits.data_ptr()
    arr[0].nb = 2
    arr[0].d_out = d_out.data_ptr()
    need = tb._lib.tb_batch_workspace_bytes(ctypes.byref(arr), 1)
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    rc = tb._lib.tb_batch_create(ctypes.byref(arr), 1, ws.data_ptr(), ws.numel(), 0, None, ctypes.byref(h))
    assert rc == tb.TB_ENOMEM


def test_autotuner_picks_a_measured_schedule(tb, tmp_path, monkeypatch):
    from paper_2608_13110_gb300 import autotune
    monkeypatch.setenv("TB_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    cands = autotune.candidate_options(16, limit=4)
    assert cands[0] == {"window_bits": 0, "bottom_bits": 0, "top_bits": 0} and len(cands) == 4
    best = autotune.tune(16, nb=4, limit=4)
    assert best in cands
    assert autotune.tune(16, nb=3, limit=4) == best  # served from the cache (same batch bucket)
    c = W.random_circuit(12, 32, None, 4, 9)
    plan = autotune.tuned_plan(c, nb=4)
    np.testing.assert_array_equal(_single(tb, plan, c.bits), _single(tb, tb.Plan.from_circuit(c, **best), c.bits))
