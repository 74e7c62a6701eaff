"""Randomised parity: seeded draws over the whole option space (qubits,
depth of either parity, window sizes, pass arithmetic, open output bits,
controlled-phase angles, Haar one-qubit gates) against the FP64 state vector,
element by element. Each draw is reproducible from its index."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

BOUND = {"fp32": 1e-5, "tf32x3": 2e-5, "bf16x3": 1.5e-4}
N_DRAWS = 40


@pytest.fixture(scope="module")
def tb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13110_gb300 import build as b
    b.build()
    import paper_2608_13110_gb300 as mod
    return mod


def draw(i):
    """The i-th configuration (plan options and circuit), from seed 50000 + i."""
    rng = np.random.default_rng(50000 + i)
    n = int(rng.integers(2, 17))
    d = int(rng.integers(2, 47))
    h = (d + 1) // 2
    prec = str(rng.choice(["fp32", "fp32", "tf32x3", "bf16x3"]))
    opts = {}
    if rng.random() < 0.5:
        opts = {"window_bits": int(rng.integers(5, 11)), "bottom_bits": int(rng.integers(5, 11)),
                "top_bits": int(rng.integers(5, 10))}
    k = 0
    if h >= 13 and n >= 3 and rng.random() < 0.4:
        k = int(rng.integers(1, min(d // 4, 10, n - 1, 6) + 1))
    ph = W.random_phases(n, d, 60000 + i) if rng.random() < 0.4 else None
    haar = rng.random() < 0.3
    return n, d, prec, opts, k, ph, haar


def all_bits(n):
    x = np.arange(1 << n)
    return ((x[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


@pytest.mark.parametrize("i", range(N_DRAWS))
def test_random_configuration(tb, oracle_mod, i):
    n, d, prec, opts, k, ph, haar = draw(i)
    if haar:
        u = W.random_unitaries(n, d, 61000 + i)
        extra = [(q, t, u[t, q]) for t in range(d + 1) for q in range(n)]
        plan_kw = dict(extra=extra)
    else:
        c = W.random_circuit(n, d, None, 0, 62000 + i)
        u = oracle_mod.circuit_gates(c)
        plan_kw = dict(cliff=c.cliff, tmask=c.tmask)
    try:
        plan = tb.Plan(n, d, precision=prec, open_k=k, cphase=ph, **opts, **plan_kw)
    except tb.TbError as e:
        # window options that do not tile this width are refused, never misplanned
        assert opts and e.status == tb.TB_EINVAL, (i, n, d, opts, e)
        plan = tb.Plan(n, d, precision=prec, open_k=k, cphase=ph, **plan_kw)
    psi = oracle_mod.sv_state(n, d, u, ph)
    rng = np.random.default_rng(63000 + i)
    if k:
        prefixes = rng.integers(0, 2, size=(3, n - k), dtype=np.uint8)
        got = plan.amplitudes(prefixes)
        y = np.arange(1 << k)
        for a in range(3):
            full = np.zeros((1 << k, n), np.uint8)
            full[:, : n - k] = prefixes[a]
            for j in range(k):
                full[:, n - k + j] = (y >> j) & 1
            ref = psi[oracle_mod.basis_index(full)]
            assert np.linalg.norm(got[a] - ref) / np.linalg.norm(ref) < BOUND[prec], (i, a)
    else:
        bits = all_bits(n) if n <= 10 else rng.integers(0, 2, size=(64, n), dtype=np.uint8)
        ref = psi[oracle_mod.basis_index(bits)]
        got = plan.amplitudes(bits)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < BOUND[prec], (i, n, d, prec, opts)
