"""Seeded synthetic inputs for open-boundary 1D brickwork circuits.

This module only draws random integers (Clifford indices, T sites, output
bitstrings). It holds none of the method's arithmetic: no gate matrices, no
contraction. Both the CUDA path and the CPU oracle read its output, and each
builds its own gate matrices from the indices.

Circuit convention (Sec. 2.1, "Bond-dimension-chi brickwork circuits"):
  * qubits q = 0..n-1 on an open chain, CZ layers l = 0..d-1;
  * layer l couples (i, i+1) for every i = l (mod 2) with i+1 < n;
  * one-qubit slots t = 0..d: slot t < d acts before CZ layer t, slot d after
    the last layer. ``cliff[t, q]`` in 0..23 is the Clifford of slot t on qubit
    q; ``tmask[t, q]`` (t < d) adds a T gate after that Clifford;
  * amplitudes psi(x) = <x|U|0^n> with ``bits[i, q] = x_q``.

The IBM instance and its experimental bitstrings are not available; these
generators stand in for them with the same shape statistics (CZ brickwork,
uniform random Cliffords on every slot, T density about 0.095 per qubit-layer,
uniform output bitstrings).
"""
from __future__ import annotations

import dataclasses

import numpy as np

N_CLIFFORD = 24
T_DENSITY = 0.095

# Indices of particular Cliffords in the table C_i = P_(i mod 4) . R_(i div 4),
# P in (I, X, Y, Z), R in (I, H, S, S.H, H.S, H.S.H).
IDX_I = 0
IDX_H = 4
DIAGONAL_CLIFFORDS = (0, 3, 8, 11)  # I, Z, S, Z.S: diagonal with (0,0) entry 1


@dataclasses.dataclass
class Circuit:
    n: int
    d: int
    cliff: np.ndarray   # (d+1, n) uint8, values 0..23
    tmask: np.ndarray   # (d, n) uint8, values 0/1
    bits: np.ndarray    # (nb, n) uint8, values 0/1
    seed: int

    @property
    def h(self) -> int:
        return (self.d + 1) // 2

    @property
    def n_t(self) -> int:
        return int(self.tmask.sum())

    def clifford_twin(self) -> "Circuit":
        """Same circuit with every T gate removed."""
        return dataclasses.replace(self, tmask=np.zeros_like(self.tmask))


def _bits(rng: np.random.Generator, nb: int, n: int) -> np.ndarray:
    return rng.integers(0, 2, size=(nb, n), dtype=np.uint8)


def random_circuit(n: int, d: int, n_t: int | None, nb: int, seed: int) -> Circuit:
    """Uniform random Clifford on every slot, exactly ``n_t`` distinct T sites
    drawn uniformly without replacement from (t, q) with t < d, and ``nb``
    uniform output bitstrings. ``n_t=None`` uses round(0.095 n d)."""
    if n_t is None:
        n_t = int(round(T_DENSITY * n * d))
    rng = np.random.default_rng(seed)
    cliff = rng.integers(0, N_CLIFFORD, size=(d + 1, n), dtype=np.uint8)
    tmask = np.zeros((d, n), dtype=np.uint8)
    if n_t > 0:
        sites = rng.choice(d * n, size=n_t, replace=False)
        tmask.reshape(-1)[sites] = 1
    bits = _bits(rng, nb, n)
    return Circuit(n, d, cliff, tmask, bits, seed)


def hdiag_circuit(n: int, d: int, n_t: int, nb: int, seed: int) -> Circuit:
    """H on every qubit at slot 0 and slot d, uniform diagonal Cliffords
    (I, Z, S, Z.S) on the interior slots, ``n_t`` T gates at uniform sites.
    Everything between the two H layers is diagonal, so these circuits have a
    closed-form amplitude at any size."""
    rng = np.random.default_rng(seed)
    cliff = np.asarray(DIAGONAL_CLIFFORDS, dtype=np.uint8)[
        rng.integers(0, len(DIAGONAL_CLIFFORDS), size=(d + 1, n))]
    cliff[0, :] = IDX_H
    cliff[d, :] = IDX_H
    tmask = np.zeros((d, n), dtype=np.uint8)
    if n_t > 0:
        sites = rng.choice(d * n, size=n_t, replace=False)
        tmask.reshape(-1)[sites] = 1
    bits = _bits(rng, nb, n)
    return Circuit(n, d, cliff, tmask, bits, seed)


def identity_circuit(n: int, d: int, nb: int, seed: int) -> Circuit:
    """Every slot holds the identity and there is no T: psi(x) = [x == 0]."""
    rng = np.random.default_rng(seed)
    bits = _bits(rng, nb, n)
    if nb > 0:
        bits[0, :] = 0
    return Circuit(n, d, np.zeros((d + 1, n), np.uint8), np.zeros((d, n), np.uint8),
                   bits, seed)


def random_unitaries(n: int, d: int, seed: int) -> np.ndarray:
    """(d+1, n, 2, 2) complex128 Haar-random one-qubit unitaries (QR of a
    complex Gaussian with the phase of R's diagonal fixed). Used to exercise
    the sweep with gates outside the Clifford+T set."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((d + 1, n, 2, 2)) + 1j * rng.standard_normal((d + 1, n, 2, 2)))
    z /= np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diagonal(r, axis1=-2, axis2=-1)
    ph = ph / np.abs(ph)
    return q * ph[..., None, :]


def random_phases(n: int, d: int, seed: int) -> np.ndarray:
    """(d, n-1) angles uniform in [0, 2 pi): one controlled-phase angle per
    (layer, pair); entries of pairs a layer does not couple are drawn too and
    ignored by both sides."""
    return np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi, size=(d, max(n - 1, 0)))


# --- The five workload shapes (seed = config_id*1000 + replica) -------------

def tiny(replica: int = 0) -> Circuit:
    """n=12, d=8, 6 T gates, 64 bitstrings (boundary width 4)."""
    return random_circuit(12, 8, 6, 64, 1000 + replica)


def scale_70_56(replica: int = 0, nb: int = 32) -> Circuit:
    """n=70, d=56, 374 T gates, 32 bitstrings (width 28, 2 GiB boundary)."""
    return random_circuit(70, 56, 374, nb, 2000 + replica)


def slice_30_40(replica: int = 1, nb: int = 32) -> Circuit:
    """n=30, d=40, 114 T gates: the oracle-sized slice of the n=70, d=56 shape."""
    return random_circuit(30, 40, 114, nb, 2000 + replica)


def batch_uneven(n_circuits: int = 64, nb: int = 32, seed0: int = 3000) -> list[Circuit]:
    """64 circuits with n ~ U[20,70], d ~ U{16,18,...,48}, T density 0.095."""
    out = []
    for i in range(n_circuits):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(20, 71))
        d = int(2 * rng.integers(8, 25))
        out.append(random_circuit(n, d, None, nb, seed0 + 100000 + i))
    return out


def precision_70_64(replica: int = 0, nb: int = 16) -> Circuit:
    """n=70, d=64, 426 T gates, 16 bitstrings (width 32, 32 GiB boundary)."""
    return random_circuit(70, 64, 426, nb, 4000 + replica)


def slice_32_48(replica: int = 1, nb: int = 16) -> Circuit:
    """n=32, d=48, 146 T gates: the oracle-sized slice of the n=70, d=64 shape."""
    return random_circuit(32, 48, 146, nb, 4000 + replica)


def serving_stream(n_requests: int, rate_hz: float = 20.0, seed: int = 5000,
                   max_width: int = 33):
    """Poisson arrivals (mean ``rate_hz``); n ~ U[16,70], d ~ U{8,10,...,2*max_width}
    (max_width 33 gives the full d <= 66 range), 1..256 uniform bitstrings per
    request. Returns a list of (arrival_time_s, Circuit)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        n = int(rng.integers(16, 71))
        d = int(2 * rng.integers(4, max_width + 1))
        nb = int(rng.integers(1, 257))
        out.append((t, random_circuit(n, d, None, nb, seed + 100000 + i)))
    return out
