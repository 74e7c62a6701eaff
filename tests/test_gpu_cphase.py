"""Controlled-phase entanglers diag(1, 1, 1, e^(i phi)) per gate (Sec. 2.1
admits any entangler of operator Schmidt rank 2; the sweep only uses its
diagonal factor). Every device path against the FP64 oracle with the same
angles: narrow plans, pass shapes, split precision, Algorithm 2 and the
closed form at n = 70."""
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


@pytest.mark.parametrize("n,d", [(2, 3), (3, 4), (5, 8), (6, 9), (9, 12), (10, 23), (13, 16)])
def test_narrow_random_unitaries_and_phases(tb, oracle_mod, n, d):
    u = W.random_unitaries(n, d, 13 * n + d)
    ph = W.random_phases(n, d, 17 * n + d)
    extra = [(q, t, u[t, q]) for t in range(d + 1) for q in range(n)]
    plan = tb.Plan(n, d, extra=extra, cphase=ph)
    bits = all_bits(n) if n <= 10 else np.random.default_rng(n).integers(0, 2, (200, n)).astype(np.uint8)
    assert rel_l2(plan.amplitudes(bits), oracle_mod.sv_amplitudes(n, d, u, bits, ph)) < TOL


@pytest.mark.parametrize("n,d,wb,bb,tt", [(6, 42, 6, 8, 5), (6, 44, 9, 8, 7), (7, 26, 5, 9, 5),
                                          (7, 26, 5, 6, 8), (6, 41, 6, 8, 5), (16, 40, 0, 0, 0),
                                          (17, 45, 0, 0, 0)])
def test_pass_schedule_vs_state_vector(tb, oracle_mod, n, d, wb, bb, tt):
    c = W.random_circuit(n, d, None, 48, 9900 + 31 * n + d)
    ph = W.random_phases(n, d, 9950 + n + d)
    plan = tb.Plan.from_circuit(c, window_bits=wb, bottom_bits=bb, top_bits=tt, cphase=ph)
    assert plan.info["n_passes"] > 0
    ref = oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), c.bits, ph)
    assert rel_l2(plan.amplitudes(c.bits), ref) < TOL


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,d", [(6, 26), (9, 29), (12, 30)])
def test_split_precision(tb, oracle_mod, prec, n, d):
    c = W.random_circuit(n, d, None, 64, 9800 + n + d)
    ph = W.random_phases(n, d, 9850 + n + d)
    ref = oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), c.bits, ph)
    got = tb.Plan.from_circuit(c, precision=prec, cphase=ph).amplitudes(c.bits)
    assert rel_l2(got, ref) < BOUND[prec]


@pytest.mark.parametrize("n,d,k", [(16, 26, 3), (15, 26, 3), (16, 25, 6), (13, 25, 1), (14, 27, 2),
                                   (5, 26, 4)])
def test_open_bits(tb, oracle_mod, n, d, k):
    """Algorithm 2: the crossing entanglers (early region and late crossings)
    and the band's own entanglers all carry their angles."""
    c = W.random_circuit(n, d, None, 0, 1300 + 10 * n + k)
    ph = W.random_phases(n, d, 7 * n + d + k)
    prefixes = np.random.default_rng(n).integers(0, 2, size=(2, n - k), dtype=np.uint8)
    got = tb.Plan.from_circuit(c, open_k=k, cphase=ph).amplitudes(prefixes)
    ref = oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), full_bits(prefixes, n, k),
                                   ph).reshape(2, -1)
    for i in range(2):
        assert rel_l2(got[i], ref[i]) < TOL


def test_pi_is_cz_bit_for_bit(tb):
    c = W.random_circuit(14, 30, None, 8, 4242)
    ph = np.full((c.d, c.n - 1), np.pi)
    a = tb.Plan.from_circuit(c).amplitudes(c.bits)
    np.testing.assert_array_equal(tb.Plan.from_circuit(c, cphase=ph).amplitudes(c.bits), a)


def _large_bits(c, oracle_mod, ph, nb, seed):
    from test_gpu_parity import _nonzero_bits
    cand = _nonzero_bits(c, oracle_mod, 64, seed)
    a = np.abs(oracle_mod.closed_form_hdiag(c, cand, ph))
    return cand[np.argsort(-a)[:nb]]


@pytest.mark.parametrize("d,prec", [(64, "fp32"), (64, "tf32x3"), (65, "fp32")])
def test_closed_form_70(tb, oracle_mod, d, prec):
    """Full n = 70 schedules (width 32 / 33) on H / diagonal / H circuits with
    random angles, against the closed form."""
    c = W.hdiag_circuit(70, d, int(round(0.095 * 70 * d)), 0, 7000 + d)
    ph = W.random_phases(70, d, 7100 + d)
    bits = _large_bits(c, oracle_mod, ph, 2, 3)
    ref = oracle_mod.closed_form_hdiag(c, bits, ph)
    got = tb.Plan.from_circuit(c, precision=prec, cphase=ph).amplitudes(bits)
    assert rel_l2(got, ref) < BOUND[prec]


def test_graph_batch_with_controlled_phases(tb):
    """Controlled-phase plans are ordinary plans for the batch runtime."""
    import torch
    circuits = [W.random_circuit(n, d, None, nb, 2100 + i)
                for i, (n, d, nb) in enumerate([(10, 27, 3), (14, 30, 2), (6, 9, 5)])]
    plans = [tb.Plan.from_circuit(c, cphase=W.random_phases(c.n, c.d, 2200 + i)) for i, c in enumerate(circuits)]
    d_bits = [torch.from_numpy(c.bits).cuda() for c in circuits]
    d_out = [torch.empty((c.bits.shape[0], 2), dtype=torch.float64, device="cuda") for c in circuits]
    batch = tb.Batch(list(zip(plans, d_bits, d_out)))
    batch.launch()
    torch.cuda.synchronize()
    for c, p, o in zip(circuits, plans, d_out):
        got = o.cpu().numpy().view(np.complex128).reshape(-1)
        np.testing.assert_array_equal(got, p.amplitudes(c.bits))
