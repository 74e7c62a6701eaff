"""Split-precision tensor-core passes (TF32X3 / BF16X3) against the FP64 oracle.

Each pass composes its paired steps into one dense complex block over 5 (TF32)
or 6 (BF16) address bits and applies it with tcgen05 MMAs as three split
products accumulated in FP32. Error bounds (relative L2 over a batch):

* TF32X3: each operand is carried to 22 significant bits (hi + lo), the
  dropped lo.lo term is 2^-22 relative, and the FP32 accumulator rounds once
  per MMA; 2e-5, twice the complex64 bar, holds at every size tested
  (measured about 1.6x the FP32 path's error).
* BF16X3: hi + lo carry 16 significant bits (2^-17 relative per operand), so
  each pass adds about 1e-5 relative error; 1.5e-4 bounds the widths tested
  here (measured 0.7e-5 .. 4e-5 up to n = 32, d = 48).
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

BOUND = {"tf32x3": 2e-5, "bf16x3": 1.5e-4}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "precision_n32_d48.json")


@pytest.fixture(scope="module")
def tb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13110_gb300 import build as b
    b.build()
    import paper_2608_13110_gb300 as mod
    mod.device_faults()  # clear
    return mod


def rel_l2(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def _amps(tb, c, bits, prec):
    return tb.Plan.from_circuit(c, precision=prec).amplitudes(bits)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,d", [(3, 26), (6, 26), (9, 28), (12, 30), (14, 34), (5, 38)])
def test_state_vector(tb, oracle_mod, prec, n, d):
    """Widths 13..19 (every window placement at bit 0, turns and row
    parities) against the dense FP64 state vector."""
    c = W.random_circuit(n, d, None, 64, 900 + n + d)
    ref = oracle_mod.sv_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), c.bits)
    got = _amps(tb, c, c.bits, prec)
    assert rel_l2(got, ref) < BOUND[prec]
    assert tb.device_faults() == 0


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_naive_boundary_30_40(tb, oracle_mod, prec):
    """Width 20 against the FP64 naive boundary contraction."""
    c = W.slice_30_40(nb=4)
    ref = oracle_mod.nb_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), c.bits)
    assert rel_l2(_amps(tb, c, c.bits, prec), ref) < BOUND[prec]


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
def test_golden_32_48(tb, prec):
    """The precision workload's oracle-sized case (n = 32, d = 48, width 24,
    146 T gates): stored FP64 amplitudes written by the oracle."""
    if not os.path.exists(GOLDEN):
        pytest.skip("golden values not generated")
    g = json.load(open(GOLDEN))
    c = W.Circuit(g["n"], g["d"], np.array(g["cliff"], np.uint8), np.array(g["tmask"], np.uint8),
                  np.array(g["bits"], np.uint8), 0)
    ref = np.array([complex(a, b) for a, b in g["amps"]])
    got = _amps(tb, c, c.bits, prec)
    assert rel_l2(got, ref) < (1e-5 if prec == "fp32" else BOUND[prec])


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_closed_form_70_64(tb, oracle_mod, prec):
    """Full n = 70, d = 64 schedule (375 / 443 dense passes over a 32 GiB
    boundary) on an H / diagonal / H circuit with a closed-form amplitude."""
    from test_gpu_parity import _nonzero_bits
    c = W.hdiag_circuit(70, 64, 426, 0, 4100)
    bits = _nonzero_bits(c, oracle_mod, 2, 1)
    ref = oracle_mod.closed_form_hdiag(c, bits)
    assert rel_l2(_amps(tb, c, bits, prec), ref) < BOUND[prec]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_clifford_twin_70_56(tb, oracle_mod, prec):
    """T gates removed: |amp|^2 is 0 or 2^-r exactly (stabilizer tableau)."""
    c = W.scale_70_56(nb=8).clifford_twin()
    got = _amps(tb, c, c.bits, prec)
    p_ref = np.array([oracle_mod.tableau_probability(c, x) for x in c.bits])
    nz = p_ref[p_ref > 0]
    assert nz.size > 0
    r = -np.log2(nz[0])
    # |a|^2 carries twice the amplitude's relative error: with the form's
    # relative-L2 bound B, |a|^2 2^r lies within 2B of 0 or 1; 4B leaves room
    # for the spread across bitstrings (TF32X3: 8e-5, BF16X3: 6e-4)
    np.testing.assert_allclose(np.abs(got) ** 2 * 2.0 ** r, p_ref * 2.0 ** r, atol=4 * BOUND[prec], rtol=0)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_deterministic_and_batch_independent(tb, prec):
    """Two calls give identical bits; a batch equals its members alone."""
    c = W.random_circuit(16, 36, None, 6, 31)
    plan = tb.Plan.from_circuit(c, precision=prec)
    a = plan.amplitudes(c.bits)
    np.testing.assert_array_equal(a, plan.amplitudes(c.bits))
    np.testing.assert_array_equal(a, np.array([plan.amplitudes(x[None])[0] for x in c.bits]))


def test_narrow_plans_use_the_fp32_kernel(tb):
    """Width <= 12 keeps the whole boundary in shared memory: no dense passes,
    same result as the default plan."""
    c = W.tiny()
    p = tb.Plan.from_circuit(c, precision="bf16x3")
    assert p.info["n_passes"] == 0
    np.testing.assert_array_equal(p.amplitudes(c.bits), tb.Plan.from_circuit(c).amplitudes(c.bits))


def test_bounded_waits_give_up_and_the_device_stays_usable(tb, oracle_mod):
    """Failure detection without a fault: the self-test's tensor-core kernels
    wait for MMAs that are never issued and its FP32 pass kernels for tile
    copies that are never issued; every wait gives up after its bounded number
    of tries, is counted (the synchronous entry returns TB_ETIMEOUT, which the
    self-test checks), and the kernels exit. Afterwards the same kernels run
    normally on the same context, in both arithmetics."""
    n_gave_up = tb.selftest_bounded_wait()
    # at least one CTA per part: the tensor-core evaluation and the FP32 passes
    assert n_gave_up >= 2
    assert tb.device_faults() == 0  # the self-test read and cleared the count
    c = W.random_circuit(9, 28, None, 8, 77)
    ref = oracle_mod.sv_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), c.bits)
    assert rel_l2(tb.Plan.from_circuit(c).amplitudes(c.bits), ref) < 1e-5
    got = tb.Plan.from_circuit(c, precision="bf16x3").amplitudes(c.bits)
    assert rel_l2(got, ref) < BOUND["bf16x3"]
    assert tb.device_faults() == 0


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_maximum_width_33(tb, oracle_mod, prec):
    """Width 33 (64 GiB boundary) with tensor-core passes, closed form."""
    from test_gpu_parity import _nonzero_bits
    c = W.hdiag_circuit(70, 66, 439, 0, 4300)
    bits = _nonzero_bits(c, oracle_mod, 1, 3)
    ref = oracle_mod.closed_form_hdiag(c, bits)
    assert rel_l2(_amps(tb, c, bits, prec), ref) < BOUND[prec]


def test_split_precision_plans_in_a_graph_batch(tb):
    """The batch runtime records tensor-core passes like any other: a mixed
    batch of FP32, 3xTF32 and 3xBF16 plans equals the single calls."""
    import torch
    circuits = [W.random_circuit(n, d, None, nb, 1800 + i)
                for i, (n, d, nb) in enumerate([(10, 28, 3), (14, 30, 2), (9, 34, 4)])]
    plans = [tb.Plan.from_circuit(c, precision=p) for c, p in zip(circuits, ("fp32", "tf32x3", "bf16x3"))]
    d_bits = [torch.from_numpy(c.bits).cuda() for c in circuits]
    d_out = [torch.empty((c.bits.shape[0], 2), dtype=torch.float64, device="cuda") for c in circuits]
    batch = tb.Batch(list(zip(plans, d_bits, d_out)))
    batch.launch()
    torch.cuda.synchronize()
    for c, p, o in zip(circuits, plans, d_out):
        got = o.cpu().numpy().view(np.complex128).reshape(-1)
        np.testing.assert_array_equal(got, p.amplitudes(c.bits))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,d", [(14, 26), (16, 30)])
def test_total_variation_of_the_output_distribution(tb, oracle_mod, prec, n, d):
    """Total variation between the output distributions of the GPU forms and
    FP64 over every bitstring (the paper compares complex64 with complex128 this
    way, Sec. 5.1). For unit vectors TV = 1/2 sum | |psi|^2 - |phi|^2 | <=
    1/2 |psi - phi| |psi + phi| <= |psi - phi|, so the relative-L2 bound of each
    form also bounds its TV."""
    c = W.random_circuit(n, d, None, 0, 1900 + n)
    x = np.arange(1 << n)
    bits = ((x[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    a = tb.Plan.from_circuit(c, precision=prec).amplitudes(bits)
    psi = oracle_mod.sv_state(n, d, oracle_mod.circuit_gates(c))
    tv = 0.5 * np.abs(np.abs(a) ** 2 - np.abs(psi) ** 2).sum()
    err = float(np.linalg.norm(a - psi))
    print(f"\nTV {prec} n={n} d={d}: {tv:.3e} (relative L2 {err:.3e})")
    assert tv <= err * (1 + 1e-9) + 1e-15
    assert err < (1e-5 if prec == "fp32" else BOUND[prec])
