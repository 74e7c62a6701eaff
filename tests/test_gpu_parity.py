"""Parity of the CUDA sweep (through the C-ABI) with the FP64 CPU oracle.

Bar: relative L2 error over each batch <= 1e-5 for complex64 (the target the
method is built to); Clifford-only twins reproduce the stabilizer |amp|^2 in
{0, 2^-r}: |amp|^2 * 2^r within 1e-4 of 0 or 1.
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


def rel_l2(a, ref):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(ref)) / np.linalg.norm(ref))


def all_bits(n):
    return np.array([[(i >> q) & 1 for q in range(n)] for i in range(1 << n)], np.uint8)


# ----------------------------------------------------------- narrow widths

def test_tiny_config_every_amplitude(tb, oracle_mod):
    """n=12, d=8 (width 4), 6 T gates: the 64 seeded bitstrings and all 4096."""
    c = W.tiny()
    u = oracle_mod.circuit_gates(c)
    plan = tb.Plan.from_circuit(c)
    got = plan.amplitudes(c.bits)
    assert rel_l2(got, oracle_mod.sv_amplitudes(c.n, c.d, u, c.bits)) < TOL
    bits = all_bits(c.n)
    got = plan.amplitudes(bits)
    ref = oracle_mod.sv_state(c.n, c.d, u)
    assert rel_l2(got, ref) < TOL
    assert abs(np.sum(np.abs(got) ** 2) - 1.0) < 1e-5


@pytest.mark.parametrize("n,d", [(2, 2), (3, 4), (4, 6), (5, 8), (7, 10), (9, 12), (10, 24), (13, 16)])
def test_narrow_random_unitaries(tb, oracle_mod, n, d):
    u = W.random_unitaries(n, d, 7 * n + d)
    extra = [(q, t, u[t, q]) for t in range(d + 1) for q in range(n)]
    plan = tb.Plan(n, d, extra=extra)
    bits = all_bits(n) if n <= 10 else np.random.default_rng(n).integers(0, 2, (200, n)).astype(np.uint8)
    assert rel_l2(plan.amplitudes(bits), oracle_mod.sv_amplitudes(n, d, u, bits)) < TOL


# ------------------------------------------------------- HBM pass schedule

# (n, d, window_bits, bottom_bits, top_bits): together these schedules use
# every pass shape with every window size it admits (5..10; 10-bit windows
# above bit 0 use rows of 64 bytes; checked on the host in
# tests/test_abi_host.py::test_pass_cases_cover_every_shape).
PASS_CASES = [
    (6, 42, 6, 8, 5), (6, 46, 8, 6, 5), (6, 36, 9, 5, 6),
    (6, 32, 5, 9, 8), (6, 36, 5, 10, 9), (7, 26, 5, 5, 9),
    (7, 26, 5, 6, 8), (7, 26, 5, 7, 7), (7, 26, 5, 8, 6), (7, 26, 5, 9, 5),
    (6, 28, 10, 5, 10), (6, 36, 10, 5, 5), (7, 28, 10, 5, 10), (6, 26, 5, 7, 7),
    (16, 40, 0, 0, 0), (17, 44, 0, 0, 0),
]


@pytest.mark.parametrize("n,d,wb,bb,tt", PASS_CASES)
def test_pass_schedule_vs_state_vector(tb, oracle_mod, n, d, wb, bb, tt):
    c = W.random_circuit(n, d, None, 48, 9000 + 31 * n + d)
    plan = tb.Plan.from_circuit(c, window_bits=wb, bottom_bits=bb, top_bits=tt)
    assert plan.info["n_passes"] > 0
    ref = oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), c.bits)
    assert rel_l2(plan.amplitudes(c.bits), ref) < TOL


@pytest.mark.parametrize("n,d,wb,bb,tt", PASS_CASES[:13])
def test_every_pass_shape_random_unitaries(tb, oracle_mod, n, d, wb, bb, tt):
    """Haar one-qubit gates on every slot: the turn passes' composed 4x4 blocks
    and every other step with dense, unstructured coefficients."""
    u = W.random_unitaries(n, d, 7 * n + d + 100 * wb + 10 * bb + tt)
    extra = [(q, t, u[t, q]) for t in range(d + 1) for q in range(n)]
    plan = tb.Plan(n, d, extra=extra, window_bits=wb, bottom_bits=bb, top_bits=tt)
    assert plan.info["n_passes"] > 0
    bits = np.random.default_rng(n + d).integers(0, 2, size=(24, n), dtype=np.uint8)
    assert rel_l2(plan.amplitudes(bits), oracle_mod.sv_amplitudes(n, d, u, bits)) < TOL


@pytest.mark.parametrize("n,d", [(8, 30), (11, 28)])
def test_pass_schedule_random_unitaries(tb, oracle_mod, n, d):
    u = W.random_unitaries(n, d, 3 * n + d)
    extra = [(q, t, u[t, q]) for t in range(d + 1) for q in range(n)]
    plan = tb.Plan(n, d, extra=extra)
    bits = all_bits(n)
    assert rel_l2(plan.amplitudes(bits), oracle_mod.sv_amplitudes(n, d, u, bits)) < TOL


def test_slice_30_40_vs_naive_boundary(tb, oracle_mod):
    """The oracle-sized slice of the n=70, d=56 workload (width 20, 114 T)."""
    c = W.slice_30_40(nb=3)
    ref = oracle_mod.nb_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), c.bits)
    got = tb.Plan.from_circuit(c).amplitudes(c.bits)
    assert rel_l2(got, ref) < TOL


# ------------------------------------------------- full-size structure pins

def test_clifford_twin_70_56_matches_tableau(tb, oracle_mod):
    """n=70, d=56 (width 28, 2 GiB boundary) with the T gates removed: every
    |amp|^2 must be 0 or 2^-r exactly as the stabilizer tableau says."""
    c = W.scale_70_56().clifford_twin()
    got = tb.Plan.from_circuit(c).amplitudes(c.bits)
    p_ref = np.array([oracle_mod.tableau_probability(c, x) for x in c.bits])
    nz = p_ref[p_ref > 0]
    assert nz.size > 0
    r = -np.log2(nz[0])
    assert np.allclose(nz, nz[0])
    v = np.abs(got) ** 2 * 2.0 ** r
    np.testing.assert_allclose(v, p_ref * 2.0 ** r, atol=1e-4, rtol=0)


def _nonzero_bits(c, oracle_mod, nb, seed):
    """Bitstrings whose closed-form amplitude has no vanishing factor."""
    tab = oracle_mod.clifford_table()
    theta = np.zeros(c.n)
    for t in range(1, c.d):
        theta += np.angle(tab[c.cliff[t].astype(int), 1, 1])
    theta += np.pi / 4 * c.tmask.sum(axis=0)
    big = (np.cos(theta) < 0).astype(np.uint8)
    rng = np.random.default_rng(seed)
    bits = np.array([np.where(rng.random(c.n) < 0.25, 1 - big, big) for _ in range(nb)], np.uint8)
    bits = np.where(np.abs(np.cos(theta / 2)) > 1e-6, bits, 1)
    return np.where(np.abs(np.sin(theta / 2)) > 1e-6, bits, 0).astype(np.uint8)


def test_closed_form_70_64(tb, oracle_mod):
    """Full n=70, d=64 schedule (width 32, 32 GiB boundary) on an H / diagonal
    / H circuit with 426 T gates, whose amplitude has a closed form."""
    c = W.hdiag_circuit(70, 64, 426, 0, 4100)
    bits = _nonzero_bits(c, oracle_mod, 3, 1)
    ref = oracle_mod.closed_form_hdiag(c, bits)
    got = tb.Plan.from_circuit(c).amplitudes(bits)
    assert rel_l2(got, ref) < TOL


def test_closed_form_70_64_tuned_schedule_batch_16(tb, oracle_mod):
    """The benchmark's launch configuration at full size: n=70, d=64, 16
    bitstrings evaluated side by side, windows of 9 bits, bottom 10, top 7 (the
    schedule the autotuner picks for width 32 on a GB300), against the closed
    form of an H / diagonal / H circuit."""
    c = W.hdiag_circuit(70, 64, 426, 0, 4100)
    bits = _nonzero_bits(c, oracle_mod, 16, 7)
    plan = tb.Plan.from_circuit(c, window_bits=9, bottom_bits=10, top_bits=7)
    assert plan.info["n_passes"] == 205
    ref = oracle_mod.closed_form_hdiag(c, bits)
    got = plan.amplitudes(bits)
    assert rel_l2(got, ref) < TOL
    # each amplitude on its own scale too (the closed form varies over decades)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-4


def test_closed_form_70_62(tb, oracle_mod):
    """d = 2 (mod 4): every edge keeps an odd number of CZ layers, so the
    amplitude is a chain sum, not a product."""
    c = W.hdiag_circuit(70, 62, 412, 2, 4200)
    ref = oracle_mod.closed_form_hdiag(c, c.bits)
    got = tb.Plan.from_circuit(c).amplitudes(c.bits)
    assert rel_l2(got, ref) < TOL


# ------------------------------------------------ API and batching behaviour

def test_batched_equals_single(tb):
    c = W.random_circuit(20, 36, None, 12, 77)
    plan = tb.Plan.from_circuit(c)
    batched = plan.amplitudes(c.bits)
    single = np.array([plan.amplitudes(x[None])[0] for x in c.bits])
    np.testing.assert_array_equal(batched, single)


def test_repeatable(tb):
    c = W.random_circuit(24, 40, None, 4, 78)
    plan = tb.Plan.from_circuit(c)
    a = plan.amplitudes(c.bits)
    b = plan.amplitudes(c.bits)
    np.testing.assert_array_equal(a, b)


def test_device_api_matches_host_api(tb):
    import torch
    for n, d in [(12, 8), (20, 34)]:
        c = W.random_circuit(n, d, None, 16, 79 + d)
        plan = tb.Plan.from_circuit(c)
        host = plan.amplitudes(c.bits)
        ws = plan.alloc_workspace(16)
        plan.upload(ws)
        d_bits = torch.from_numpy(c.bits).cuda()
        d_out = torch.empty((16, 2), dtype=torch.float64, device="cuda")
        plan.amplitudes_device(d_bits, ws, d_out)
        torch.cuda.synchronize()
        dev = d_out.cpu().numpy().view(np.complex128).reshape(-1)
        np.testing.assert_array_equal(dev, host)


def test_small_workspace_runs_one_boundary_at_a_time(tb):
    import torch
    c = W.random_circuit(15, 30, None, 5, 80)
    plan = tb.Plan.from_circuit(c)
    full = plan.amplitudes(c.bits)
    need = plan.workspace_min_bytes() + 4096
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    np.testing.assert_array_equal(plan.amplitudes(c.bits, ws=ws), full)
    tiny = torch.empty(plan.workspace_min_bytes() // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(tb.TbError) as e:
        plan.amplitudes(c.bits, ws=tiny)
    assert e.value.status == tb.TB_ENOMEM


def test_edge_cases(tb, oracle_mod):
    # no bitstrings
    plan = tb.Plan(10, 30)
    assert plan.amplitudes(np.zeros((0, 10), np.uint8)).size == 0
    # identity circuit: psi(x) = [x == 0], narrow and wide
    for n, d in [(9, 10), (9, 30)]:
        c = W.identity_circuit(n, d, 6, 5)
        got = tb.Plan.from_circuit(c).amplitudes(c.bits)
        exp = np.array([1.0 if not x.any() else 0.0 for x in c.bits])
        np.testing.assert_allclose(got, exp, atol=1e-6)
    # two qubits: no absorbed middle row, narrow and wide
    for d in (6, 28):
        c = W.random_circuit(2, d, None, 4, 90 + d)
        ref = oracle_mod.sv_amplitudes(2, d, oracle_mod.circuit_gates(c), all_bits(2))
        assert rel_l2(tb.Plan.from_circuit(c).amplitudes(all_bits(2)), ref) < TOL


def test_maximum_width_33_closed_form(tb, oracle_mod):
    """The widest boundary the device path evaluates: n = 70, d = 66, width 33
    (2^33 complex64 = 64 GiB), against the exact amplitude of an H / diagonal /
    H circuit (d = 2 mod 4: a chain sum)."""
    c = W.hdiag_circuit(70, 66, 439, 0, 4300)
    bits = _nonzero_bits(c, oracle_mod, 1, 3)
    plan = tb.Plan.from_circuit(c)
    assert plan.info["boundary_bits"] == 33
    ref = oracle_mod.closed_form_hdiag(c, bits)
    assert rel_l2(plan.amplitudes(bits), ref) < TOL


def test_maximum_width_35_closed_form(tb, oracle_mod):
    """The widest boundary the device path evaluates: n = d = 70, width 35
    (2^35 complex64 = 256 GiB: the paper's largest intermediate) in one GPU's
    HBM, windows 10 / bottom 10 / top 9 (10-bit windows above address bit 0
    at full size), against the exact amplitude of an H / diagonal / H
    circuit."""
    import torch
    c = W.hdiag_circuit(70, 70, 468, 0, 4350)
    bits = _nonzero_bits(c, oracle_mod, 1, 9)
    plan = tb.Plan.from_circuit(c, window_bits=10, bottom_bits=10, top_bits=9)
    assert plan.info["boundary_bits"] == 35
    torch.cuda.empty_cache()
    if torch.cuda.mem_get_info()[0] < plan.workspace_bytes(1) + (2 << 30):
        pytest.skip("the device has no room for a 2^35-entry boundary")
    try:
        got = plan.amplitudes(bits)
    finally:
        torch.cuda.empty_cache()
    assert rel_l2(got, oracle_mod.closed_form_hdiag(c, bits)) < TOL
