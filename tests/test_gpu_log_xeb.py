"""FP64 log-XEB reduction on the device (Sec. 5.2, normalized log-XEB
estimator) against the oracle's estimator, through the C-ABI."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def tb(torch):
    from paper_2608_13110_gb300 import build as b
    b.build()
    import paper_2608_13110_gb300 as mod
    return mod


def _device_xeb(tb, torch, amps, n):
    d_amps = torch.from_numpy(np.ascontiguousarray(amps.astype(np.complex128)).view(np.float64).reshape(-1, 2)).cuda()
    d_out = torch.empty(1, dtype=torch.float64, device="cuda")
    tb.log_xeb_device(d_amps, n, d_out)
    torch.cuda.synchronize()
    return float(d_out.cpu()[0])


@pytest.mark.parametrize("nb", [1, 1023, 20000, 100003])
def test_porter_thomas_draws(tb, torch, oracle_mod, nb):
    """Amplitudes with Porter-Thomas weights (2^n |a|^2 ~ Exp(1)): the
    estimator is near 0 and device and oracle agree to 1e-12."""
    rng = np.random.default_rng(700 + nb)
    n = 40
    z = (rng.normal(size=nb) + 1j * rng.normal(size=nb)) * np.sqrt(0.5 / 2.0 ** n)
    got = _device_xeb(tb, torch, z, n)
    ref = oracle_mod.log_xeb(z, n)
    assert abs(got - ref) < 1e-12
    if nb >= 20000:
        assert abs(ref) < 5 * 1.28 / np.sqrt(nb)


def test_uniform_distribution_gives_gamma(tb, torch, oracle_mod):
    """|a|^2 = 2^-n for every amplitude: F = gamma exactly (up to rounding)."""
    n = 16
    z = np.full(1 << 14, 2.0 ** (-n / 2), np.complex128)
    got = _device_xeb(tb, torch, z, n)
    assert abs(got - np.euler_gamma) < 1e-12
    assert abs(got - oracle_mod.log_xeb(z, n)) < 1e-12


def test_zero_amplitude_gives_minus_infinity(tb, torch):
    z = np.full(12000, 0.01 + 0.02j, np.complex128)
    z[4567] = 0.0
    got = _device_xeb(tb, torch, z, 30)
    assert np.isneginf(got)


def test_on_the_sweep_output(tb, torch, oracle_mod):
    """The reduction enqueued after tb_amplitudes_device on the same stream,
    over the sweep's own output (n=30, d=40 slice), equals the oracle's
    estimator of the same amplitudes, and the amplitudes themselves match the
    naive-boundary oracle."""
    c = W.slice_30_40(nb=2)
    more = np.repeat(c.bits, 6000, axis=0)
    more[::3, 0] ^= 1
    bits = np.concatenate([c.bits, more])  # the first two rows are the slice's own bitstrings
    plan = tb.Plan.from_circuit(c)
    ws = plan.alloc_workspace(bits.shape[0])
    plan.upload(ws)
    d_bits = torch.from_numpy(bits).cuda()
    d_out = torch.empty((bits.shape[0], 2), dtype=torch.float64, device="cuda")
    f = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    plan.amplitudes_device(d_bits, ws, d_out, st)
    tb.log_xeb_device(d_out, c.n, f, st)
    torch.cuda.synchronize()
    amps = d_out.cpu().numpy().view(np.complex128).reshape(-1)
    assert abs(float(f.cpu()[0]) - oracle_mod.log_xeb(amps, c.n)) < 1e-12
    ref = oracle_mod.nb_amplitudes(c.n, c.d, oracle_mod.circuit_gates(c), c.bits)
    assert np.linalg.norm(amps[:2] - ref) / np.linalg.norm(ref) < 1e-5
