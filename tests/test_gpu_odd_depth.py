"""Odd circuit depth (Proposition 1's turn case) on the device path.

With d odd the layers that couple an odd row to the next one number
ceil(d/2) - 1: a forward row's last step sums the row out (its top address
bit becomes 0) and the next, backward row's first step creates the value of
layer d - 1 in that bit. The boundary keeps width ceil(d/2) and every kernel
runs the two steps as ordinary controlled 2x2 steps. These tests compare the
odd-depth paths with the FP64 oracle element by element: narrow plans, every
HBM pass shape, the split-precision passes, open output bits with crossing
layers of both parities, and full-size structure pins.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
BOUND = {"fp32": 1e-5, "tf32x3": 2e-5, "bf16x3": 1.5e-4}


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
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def all_bits(n):
    x = np.arange(1 << n)
    return ((x[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def full_bits(prefixes, n, k):
    na = prefixes.shape[0]
    out = np.zeros((na, 1 << k, n), np.uint8)
    out[:, :, : n - k] = prefixes[:, None, :]
    y = np.arange(1 << k)
    for j in range(k):
        out[:, :, n - k + j] = (y >> j) & 1
    return out.reshape(-1, n)


@pytest.mark.parametrize("n,d", [(2, 3), (3, 5), (4, 7), (5, 9), (6, 3), (7, 11), (9, 13), (10, 23), (13, 15)])
def test_narrow_random_unitaries(tb, oracle_mod, n, d):
    """Widths 2..12 (one CTA holds the boundary), Haar one-qubit gates, both
    parities of the last absorbed row."""
    u = W.random_unitaries(n, d, 11 * n + d)
    extra = [(q, t, u[t, q]) for t in range(d + 1) for q in range(n)]
    plan = tb.Plan(n, d, extra=extra)
    assert plan.info["boundary_bits"] == (d + 1) // 2
    bits = all_bits(n) if n <= 10 else np.random.default_rng(n).integers(0, 2, (200, n)).astype(np.uint8)
    assert rel_l2(plan.amplitudes(bits), oracle_mod.sv_amplitudes(n, d, u, bits)) < TOL


# window, bottom and top widths chosen so that the sum-out / create step sits
# in every pass shape (bottom, top, forward and reversed windows, turns)
ODD_PASS_CASES = [
    (6, 41, 6, 8, 5), (6, 45, 8, 6, 5), (6, 35, 9, 5, 6), (6, 43, 9, 8, 7),
    (7, 25, 5, 6, 8), (7, 25, 5, 5, 9), (7, 25, 5, 9, 5), (16, 39, 0, 0, 0), (17, 45, 0, 0, 0),
    (5, 33, 0, 0, 0),
]


@pytest.mark.parametrize("n,d,wb,bb,tt", ODD_PASS_CASES)
def test_pass_schedule_vs_state_vector(tb, oracle_mod, n, d, wb, bb, tt):
    c = W.random_circuit(n, d, None, 48, 9500 + 31 * n + d)
    plan = tb.Plan.from_circuit(c, window_bits=wb, bottom_bits=bb, top_bits=tt)
    assert plan.info["n_passes"] > 0
    ref = oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), c.bits)
    assert rel_l2(plan.amplitudes(c.bits), ref) < TOL


@pytest.mark.parametrize("n,d", [(8, 29), (11, 27)])
def test_pass_schedule_random_unitaries(tb, oracle_mod, n, d):
    u = W.random_unitaries(n, d, 5 * n + d)
    extra = [(q, t, u[t, q]) for t in range(d + 1) for q in range(n)]
    bits = all_bits(n)
    got = tb.Plan(n, d, extra=extra).amplitudes(bits)
    assert rel_l2(got, oracle_mod.sv_amplitudes(n, d, u, bits)) < TOL


def test_naive_boundary_30_41(tb, oracle_mod):
    """n = 30, d = 41 (width 21) against the FP64 naive boundary contraction."""
    c = W.random_circuit(30, 41, None, 3, 4141)
    ref = oracle_mod.nb_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), c.bits)
    assert rel_l2(tb.Plan.from_circuit(c).amplitudes(c.bits), ref) < TOL


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,d", [(3, 25), (6, 27), (9, 29), (12, 31), (5, 37)])
def test_split_precision_vs_state_vector(tb, oracle_mod, prec, n, d):
    c = W.random_circuit(n, d, None, 64, 9700 + n + d)
    ref = oracle_mod.sv_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), c.bits)
    got = tb.Plan.from_circuit(c, precision=prec).amplitudes(c.bits)
    assert rel_l2(got, ref) < BOUND[prec]
    assert tb.device_faults() == 0


@pytest.mark.parametrize("n,d,k", [(16, 25, 3), (15, 25, 3), (16, 27, 6), (13, 25, 1), (14, 25, 2),
                                   (15, 29, 5), (5, 25, 4), (4, 25, 3), (17, 27, 5)])
def test_open_bits_vs_state_vector(tb, oracle_mod, n, d, k):
    """Algorithm 2 with d odd: crossing layers even (the boundary's h bits all
    cross) and odd (h - 1 crossings; the top bit stays 0)."""
    c = W.random_circuit(n, d, None, 0, 1300 + 10 * n + k)
    prefixes = np.random.default_rng(n).integers(0, 2, size=(2, n - k), dtype=np.uint8)
    plan = tb.Plan.from_circuit(c, open_k=k)
    got = plan.amplitudes(prefixes)
    ref = oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), full_bits(prefixes, n, k)).reshape(2, -1)
    for i in range(2):
        assert rel_l2(got[i], ref[i]) < TOL


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_open_bits_split_precision(tb, oracle_mod, prec):
    c = W.random_circuit(15, 27, None, 0, 1450)
    k = 4
    prefixes = np.random.default_rng(6).integers(0, 2, size=(2, 11), dtype=np.uint8)
    got = tb.Plan.from_circuit(c, open_k=k, precision=prec).amplitudes(prefixes)
    ref = oracle_mod.sv_amplitudes(15, 27, oracle_mod.circuit_gates(c), full_bits(prefixes, 15, k)).reshape(2, -1)
    assert rel_l2(got.reshape(-1), ref.reshape(-1)) < BOUND[prec]


def _large_bits(c, oracle_mod, nb, seed):
    """nb of 64 candidate bitstrings (no vanishing one-qubit factor) with the
    largest closed-form amplitudes: d odd leaves a CZ on every other edge,
    whose pair factors can cancel too."""
    from test_gpu_parity import _nonzero_bits
    cand = _nonzero_bits(c, oracle_mod, 64, seed)
    a = np.abs(oracle_mod.closed_form_hdiag(c, cand))
    return cand[np.argsort(-a)[:nb]]


def test_clifford_twin_70_55_matches_tableau(tb, oracle_mod):
    """n = 70, d = 55 (width 28) with no T gate: |amp|^2 is 0 or 2^-r exactly."""
    c = W.random_circuit(70, 55, 0, 8, 5555)
    got = tb.Plan.from_circuit(c).amplitudes(c.bits)
    p_ref = np.array([oracle_mod.tableau_probability(c, x) for x in c.bits])
    nz = p_ref[p_ref > 0]
    assert nz.size > 0
    r = -np.log2(nz[0])
    assert np.allclose(nz, nz[0])
    np.testing.assert_allclose(np.abs(got) ** 2 * 2.0 ** r, p_ref * 2.0 ** r, atol=1e-4, rtol=0)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
def test_closed_form_70_63(tb, oracle_mod, prec):
    """Full n = 70, d = 63 schedule (width 32, 32 GiB boundary) on an H /
    diagonal / H circuit whose amplitude has a closed form."""
    c = W.hdiag_circuit(70, 63, 419, 0, 6300)
    bits = _large_bits(c, oracle_mod, 2, 1)
    ref = oracle_mod.closed_form_hdiag(c, bits)
    assert rel_l2(tb.Plan.from_circuit(c, precision=prec).amplitudes(bits), ref) < BOUND[prec]


def test_maximum_width_33_odd_depth(tb, oracle_mod):
    """n = 70, d = 65: the widest odd-depth boundary (2^33 entries), closed
    form, and the open plan of the same circuit (k = 8, crossing layers odd
    since n - k - 1 = 61) on one prefix."""
    c = W.hdiag_circuit(70, 65, 432, 0, 6500)
    bits = _large_bits(c, oracle_mod, 1, 4)
    plan = tb.Plan.from_circuit(c)
    assert plan.info["boundary_bits"] == 33
    assert rel_l2(plan.amplitudes(bits), oracle_mod.closed_form_hdiag(c, bits)) < TOL
    k = 8
    got = tb.Plan.from_circuit(c, open_k=k).amplitudes(bits[:, : c.n - k])[0]
    ref = oracle_mod.closed_form_hdiag(c, full_bits(bits[:, : c.n - k], c.n, k))
    assert rel_l2(got, ref) < TOL


def test_odd_and_even_depth_plans_in_one_graph_batch(tb):
    import torch
    circuits = [W.random_circuit(n, d, None, nb, 2000 + i)
                for i, (n, d, nb) in enumerate([(10, 27, 3), (14, 30, 2), (9, 33, 4), (6, 9, 5)])]
    plans = [tb.Plan.from_circuit(c) for c in circuits]
    d_bits = [torch.from_numpy(c.bits).cuda() for c in circuits]
    d_out = [torch.empty((c.bits.shape[0], 2), dtype=torch.float64, device="cuda") for c in circuits]
    batch = tb.Batch(list(zip(plans, d_bits, d_out)))
    batch.launch()
    torch.cuda.synchronize()
    for c, p, o in zip(circuits, plans, d_out):
        got = o.cpu().numpy().view(np.complex128).reshape(-1)
        np.testing.assert_array_equal(got, p.amplitudes(c.bits))
