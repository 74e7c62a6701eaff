"""Open output bits (Algorithm 2): one evaluation returns the 2^k amplitudes
<a, b|U|0^n> of a prefix a, compared with the plain definition (FP64 state
vector or naive boundary) element by element."""
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


def full_bits(prefixes, n, k):
    """Every (a, b) bitstring, row-major over (prefix, y), b_j = bit j of y."""
    na = prefixes.shape[0]
    out = np.zeros((na, 1 << k, n), np.uint8)
    out[:, :, : n - k] = prefixes[:, None, :]
    y = np.arange(1 << k)
    for j in range(k):
        out[:, :, n - k + j] = (y >> j) & 1
    return out.reshape(-1, n)


def rel_l2(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("n,d,k", [(16, 26, 3), (16, 26, 6), (13, 26, 1), (15, 28, 5), (14, 30, 7),
                                   (17, 26, 2), (5, 26, 4), (4, 26, 3)])
def test_state_vector(tb, oracle_mod, n, d, k):
    """Widths 13..15, both parities of the crossing layers (n-k-1 even and
    odd), k = 1..7, and fixed regions of a single row (n - k = 1)."""
    c = W.random_circuit(n, d, None, 0, 1300 + 10 * n + k)
    rng = np.random.default_rng(n * 100 + k)
    prefixes = rng.integers(0, 2, size=(3, n - k), dtype=np.uint8)
    plan = tb.Plan.from_circuit(c, open_k=k)
    assert plan.info["open_width"] == (d + 1) // 2  # Proposition 2: width ceil(d/2)
    got = plan.amplitudes(prefixes)
    assert got.shape == (3, 1 << k)
    ref = oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), full_bits(prefixes, n, k)).reshape(3, -1)
    for i in range(3):
        assert rel_l2(got[i], ref[i]) < TOL


def test_naive_boundary_sampled_30_40(tb, oracle_mod):
    """n = 30, d = 40 (width 20), k = 8: 256 amplitudes per prefix; eight
    sampled suffixes per prefix against the FP64 naive boundary."""
    c = W.slice_30_40(nb=0)
    k = 8
    rng = np.random.default_rng(5)
    prefixes = rng.integers(0, 2, size=(2, c.n - k), dtype=np.uint8)
    got = tb.Plan.from_circuit(c, open_k=k).amplitudes(prefixes)
    ys = rng.choice(1 << k, size=8, replace=False)
    bits = full_bits(prefixes, c.n, k).reshape(2, 1 << k, c.n)[:, ys, :].reshape(-1, c.n)
    ref = oracle_mod.nb_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), bits).reshape(2, -1)
    assert rel_l2(got[:, ys].reshape(-1), ref.reshape(-1)) < TOL


def test_matches_the_plain_sweep_at_70_56(tb):
    """n = 70, d = 56 (width 28), k = 8: the open plan's batch equals the
    single-amplitude sweep on the same bitstrings."""
    c = W.scale_70_56(nb=0)
    k = 8
    prefix = np.random.default_rng(9).integers(0, 2, size=(1, c.n - k), dtype=np.uint8)
    got = tb.Plan.from_circuit(c, open_k=k).amplitudes(prefix)[0]
    ys = np.array([0, 1, 37, 128, 255])
    bits = full_bits(prefix, c.n, k)[ys]
    ref = tb.Plan.from_circuit(c).amplitudes(bits)
    assert rel_l2(got[ys], ref) < TOL
    # the batch is a conditional distribution's support: Q_a > 0
    assert np.sum(np.abs(got) ** 2) > 0


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_split_precision_sweep(tb, oracle_mod, prec):
    c = W.random_circuit(16, 28, None, 0, 1400)
    k = 4
    prefixes = np.random.default_rng(3).integers(0, 2, size=(2, 12), dtype=np.uint8)
    got = tb.Plan.from_circuit(c, open_k=k, precision=prec).amplitudes(prefixes)
    ref = oracle_mod.sv_amplitudes(16, 28, oracle_mod.circuit_gates(c), full_bits(prefixes, 16, k)).reshape(2, -1)
    assert rel_l2(got.reshape(-1), ref.reshape(-1)) < (2e-5 if prec == "tf32x3" else 1.5e-4)


def test_device_entry_and_batch_split(tb):
    """Device-resident prefixes; a workspace for one prefix evaluates many in
    turn with the same result."""
    import torch
    c = W.random_circuit(20, 30, None, 0, 1500)
    k = 5
    plan = tb.Plan.from_circuit(c, open_k=k)
    prefixes = np.random.default_rng(4).integers(0, 2, size=(5, 15), dtype=np.uint8)
    ws = torch.empty(plan.workspace_min_bytes(), dtype=torch.uint8, device="cuda")
    plan.upload(ws)
    d_out = torch.empty((5 << k, 2), dtype=torch.float64, device="cuda")
    plan.amplitudes_device(torch.from_numpy(prefixes).cuda(), ws, d_out)
    torch.cuda.synchronize()
    dev = d_out.cpu().numpy().view(np.complex128).reshape(5, -1)
    np.testing.assert_array_equal(dev, plan.amplitudes(prefixes))


def test_open_plans_are_rejected_elsewhere(tb):
    import torch
    c = W.random_circuit(16, 26, None, 0, 1600)
    plan = tb.Plan.from_circuit(c, open_k=3)
    with pytest.raises(tb.TbError) as e:
        plan.amplitudes_noalloc(torch.zeros((1, 13), dtype=torch.uint8, device="cuda"),
                                torch.empty((8, 2), dtype=torch.float64, device="cuda"))
    assert e.value.status == tb.TB_EINVAL
    with pytest.raises(tb.TbError):
        plan.amplitudes(np.full((1, 13), 2, np.uint8))


def test_maximum_width_33_every_suffix(tb, oracle_mod):
    """n = 70, d = 66 (width 33: a 64 GiB boundary and a 32 GiB late-region
    buffer), k = 8: all 256 amplitudes of a prefix against the closed form of
    an H / diagonal / H circuit."""
    from test_gpu_parity import _nonzero_bits
    c = W.hdiag_circuit(70, 66, 439, 0, 4300)
    k = 8
    prefix = _nonzero_bits(c, oracle_mod, 1, 5)[:, : c.n - k]
    got = tb.Plan.from_circuit(c, open_k=k).amplitudes(prefix)[0]
    ref = oracle_mod.closed_form_hdiag(c, full_bits(prefix, c.n, k))
    assert rel_l2(got, ref) < TOL


@pytest.mark.parametrize("k,join", [(1, "fp32"), (3, "fp32"), (4, "slices"), (4, "fp32"), (6, "slices"),
                                    (8, "slices"), (8, "fp32"), (10, "slices"), (10, "fp32")])
def test_in_place_join_and_crossings(tb, oracle_mod, k, join):
    """An HBM budget below two boundaries makes the plan work in place: the
    join in row slices on the tensor cores through a scratch of one slice
    (or, when the budget cannot hold that, in FP32 over the boundary itself)
    and late crossings that write each output row over its first input row
    (rows at doubling strides). n = 16, d = 40 (width 20), three prefixes,
    every suffix against the state vector."""
    c = W.random_circuit(16, 40, None, 0, 4700 + k)
    rng = np.random.default_rng(4800 + k)
    prefixes = rng.integers(0, 2, size=(3, 16 - k), dtype=np.uint8)
    # 12 MiB: the 8 MiB boundary and a join slice fit, a second boundary does
    # not; 8 MiB + 64 KiB: the boundary and the rescaling state only
    budget = (12 << 20) if join == "slices" else (8 << 20) + (64 << 10)
    plan = tb.Plan.from_circuit(c, open_k=k, hbm_budget_bytes=budget)
    scratch = (max(128, (1 << (20 - k)) >> 6) << (k + 3)) if join == "slices" else 0
    assert tb.Plan.from_circuit(c, open_k=k).workspace_bytes(1) - plan.workspace_bytes(1) == (8 << 20) - scratch
    got = plan.amplitudes(prefixes)
    ref = oracle_mod.sv_amplitudes(16, 40, oracle_mod.circuit_gates(c), full_bits(prefixes, 16, k)).reshape(3, -1)
    for i in range(3):
        assert rel_l2(got[i], ref[i]) < TOL


def test_maximum_width_35_in_place(tb, oracle_mod):
    """n = d = 70, k = 8: the paper's contraction (Sec. 5: width 35, 256
    amplitudes per prefix) on one GPU, in place (a 256 GiB boundary); every
    suffix of a prefix against the closed form of an H / diagonal / H
    circuit with the same T count (468)."""
    import torch
    from test_gpu_parity import _nonzero_bits
    c = W.hdiag_circuit(70, 70, 468, 0, 4900)
    k = 8
    plan = tb.Plan.from_circuit(c, open_k=k)
    assert plan.info["boundary_bits"] == 35
    need = plan.workspace_bytes(1)
    assert need < (8 << 35) + (5 << 30)  # one boundary and a 4 GiB join slice: the plan works in place
    torch.cuda.empty_cache()  # blocks cached by the earlier tests of this process
    if torch.cuda.mem_get_info()[0] < need + (2 << 30):
        pytest.skip("the device has no room for a 2^35-entry boundary")
    prefix = _nonzero_bits(c, oracle_mod, 1, 7)[:, : c.n - k]
    try:
        got = plan.amplitudes(prefix)[0]
    finally:
        torch.cuda.empty_cache()  # hand the 256 GiB back for the tests that allocate outside PyTorch
    ref = oracle_mod.closed_form_hdiag(c, full_bits(prefix, c.n, k))
    assert rel_l2(got, ref) < TOL


def test_batched_sampling_draws_from_the_conditional(tb, oracle_mod):
    """Sec. 4 sampler end to end: for every draw, the prefix is the caller's
    uniform draw and the suffix is the inverse of p(. | a) (from the FP64 state
    vector) at the caller's uniform variate."""
    n, d, k = 14, 26, 4
    c = W.random_circuit(n, d, None, 0, 1700)
    plan = tb.Plan.from_circuit(c, open_k=k)
    bits, amps, q = tb.sample(plan, 12, np.random.default_rng(11))
    rng = np.random.default_rng(11)  # replay the same variates
    prefixes = rng.integers(0, 2, size=(12, n - k), dtype=np.uint8)
    u = rng.random(12)
    np.testing.assert_array_equal(bits[:, : n - k], prefixes)
    psi = oracle_mod.sv_state(n, d, oracle_mod.circuit_gates(c))
    idx = oracle_mod.basis_index(full_bits(prefixes, n, k)).reshape(12, -1)
    p = np.abs(psi[idx]) ** 2
    np.testing.assert_allclose(q, p.sum(axis=1), rtol=1e-4)
    cdf = np.cumsum(p, axis=1) / p.sum(axis=1, keepdims=True)
    for i in range(12):
        b = int(oracle_mod.basis_index(bits[i:i + 1, n - k:])[0])
        lo = cdf[i, b - 1] if b > 0 else 0.0
        assert lo - 1e-4 <= u[i] <= cdf[i, b] + 1e-4
        assert abs(amps[i] - psi[oracle_mod.basis_index(bits[i:i + 1])[0]]) < 1e-5 * np.abs(psi).max() + 1e-6


def test_closed_form_70_64_in_the_benchmark_launch(tb, oracle_mod):
    """The open workload's launch configuration at full size: n = 70, d = 64,
    k = 8, two prefixes side by side, windows 9 / bottom 10 / top 7 (the
    autotuner's choice at width 32): every suffix of both prefixes against the
    closed form of an H / diagonal / H circuit."""
    from test_gpu_parity import _nonzero_bits
    c = W.hdiag_circuit(70, 64, 426, 0, 4100)
    k = 8
    prefixes = _nonzero_bits(c, oracle_mod, 2, 11)[:, : c.n - k]
    plan = tb.Plan.from_circuit(c, open_k=k, window_bits=9, bottom_bits=10, top_bits=7)
    got = plan.amplitudes(prefixes)
    ref = oracle_mod.closed_form_hdiag(c, full_bits(prefixes, c.n, k)).reshape(2, -1)
    for a in range(2):
        assert rel_l2(got[a], ref[a]) < TOL


@pytest.mark.parametrize("k", [9, 10])
def test_tensor_core_join_at_its_largest(tb, oracle_mod, k):
    """k = 9 and 10 (the join is a 512^2 / 1024^2 complex matrix product on the
    tensor cores, 3xTF32): n = 30, d = 40 (width 20), two prefixes, six
    sampled suffixes each against the FP64 naive boundary, and every suffix
    against the state vector of an n = 16, d = 40 circuit."""
    c = W.slice_30_40(nb=0)
    rng = np.random.default_rng(4400 + k)
    prefixes = rng.integers(0, 2, size=(2, c.n - k), dtype=np.uint8)
    got = tb.Plan.from_circuit(c, open_k=k).amplitudes(prefixes)
    ys = rng.choice(1 << k, size=6, replace=False)
    for i in range(2):
        bits = full_bits(prefixes[i:i + 1], c.n, k)[ys]
        ref = oracle_mod.nb_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), bits)
        assert rel_l2(got[i, ys], ref) < TOL
    c2 = W.random_circuit(16, 40, None, 0, 4500 + k)
    pre2 = rng.integers(0, 2, size=(2, 16 - k), dtype=np.uint8)
    got2 = tb.Plan.from_circuit(c2, open_k=k).amplitudes(pre2)
    ref2 = oracle_mod.sv_amplitudes(16, 40, oracle_mod.circuit_gates(c2), full_bits(pre2, 16, k)).reshape(2, -1)
    for i in range(2):
        assert rel_l2(got2[i], ref2[i]) < TOL
