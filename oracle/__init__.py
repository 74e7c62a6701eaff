"""FP64 CPU oracle for exact brickwork-circuit amplitudes.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. The product
path (the CUDA library and its binding) never imports, links or calls it, and
this package never imports the product. The only module both sides read is the
seeded input generator ``workloads``, which holds no arithmetic of the method.

What it computes (the paper's amplitude, Sec. 2.2): psi(x) = <x|U|0^n> for an
open 1D brickwork circuit with CZ entanglers (Sec. 2.1), in several independent
ways:

* ``sv_state`` / ``sv_amplitudes`` -- dense state vector, gate by gate (C);
* ``nb_amplitudes`` -- naive row-by-row contraction of the circuit's tensor
  network (Sec. 2.2 mapping; every row absorbed in forward time with an explicit
  wire index; no snake order, slot reuse, fusion or rescaling) (C);
* ``feynman_amplitude`` -- brute-force sum over every CZ-layer value (C);
* ``kron_state`` -- product of full 2^n x 2^n layer matrices (numpy);
* ``tableau_probability`` -- |psi|^2 of Clifford-only circuits from an
  Aaronson-Gottesman stabilizer tableau (C);
* ``closed_form_hdiag`` -- closed form for circuits whose first and last slots
  are H on every qubit and whose interior slots are diagonal (numpy);
* ``log_xeb`` -- the log-XEB estimator of Sec. 5.2 (numpy);
* ``alg1_cost`` -- contraction width W and cost log2 C of Algorithm 1's path
  (Sec. 2.2 cost definitions, Sec. 3.1), counted over the network's legs
  (pure Python).

Readings of points the paper leaves open (also listed in the design notes):
d+1 one-qubit slots, slot t < d before CZ layer t; U_(q,t) = T^tau . C (the
Clifford acts first); T = diag(1, e^(i pi/4)); the 24 Cliffords are
C_k = P_(k mod 4) . R_(k div 4) with P in (I, X, Y, Z), Y = [[0,-i],[i,0]],
R in (I, H, S, S.H, H.S, H.S.H); layer l couples (i, i+1) for i = l (mod 2).

Pins: see tests/test_oracle_pins.py (brute force, Kronecker product, norm,
tableau, closed form, identity circuit, the paper's printed (W, log2 C) and
Proposition 1's width). Every function here is pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tbo.c")
_LIB_PATH = os.path.join(_HERE, "libtbo.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC,
               "-o", _LIB_PATH + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.tbo_sv_state.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_void_p, dp]
        lib.tbo_nb_amplitude.argtypes = [ctypes.c_int, ctypes.c_int, dp, u8p, dp, ip]
        lib.tbo_feynman.argtypes = [ctypes.c_int, ctypes.c_int, dp, u8p, dp]
        lib.tbo_tableau_prob.argtypes = [ctypes.c_int, ctypes.c_int, u8p, u8p, dp]
        lib.tbo_num_threads.argtypes = []
        lib.tbo_set_num_threads.argtypes = [ctypes.c_int]
        for f in ("tbo_sv_state", "tbo_nb_amplitude", "tbo_feynman", "tbo_tableau_prob",
                  "tbo_num_threads", "tbo_set_num_threads"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the C oracle uses."""
    return int(_load().tbo_num_threads())


def set_num_threads(t: int) -> int:
    """Use t OpenMP threads from now on (t >= 1); returns the count in effect."""
    return int(_load().tbo_set_num_threads(int(t)))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


# --------------------------------------------------------------------------
# Gate matrices (the oracle's own construction)
# --------------------------------------------------------------------------

_SQ2 = np.sqrt(0.5)
_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_H = _SQ2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)
_S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
T_GATE = np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128)


def clifford_table() -> np.ndarray:
    """(24, 2, 2) complex128: C_k = P_(k mod 4) @ R_(k div 4)."""
    paulis = (_I2, _X, _Y, _Z)
    rots = (_I2, _H, _S, _S @ _H, _H @ _S, _H @ _S @ _H)
    return np.array([paulis[k % 4] @ rots[k // 4] for k in range(24)])


def gates(cliff: np.ndarray, tmask: np.ndarray, extra=None) -> np.ndarray:
    """(d+1, n, 2, 2) complex128 slot gates U_(q,t) = T^tau . C_(cliff) [. extra].

    ``extra`` is an optional (d+1, n, 2, 2) array applied after the Clifford
    and T of each slot (None = identity)."""
    cliff = np.asarray(cliff)
    tmask = np.asarray(tmask)
    d1, n = cliff.shape
    tab = clifford_table()
    u = tab[cliff.astype(np.int64)]
    tm = np.zeros((d1, n), dtype=bool)
    tm[: d1 - 1] = tmask.astype(bool)
    u = np.where(tm[..., None, None], np.einsum("ab,tqbc->tqac", T_GATE, u), u)
    if extra is not None:
        u = np.einsum("tqab,tqbc->tqac", np.asarray(extra, np.complex128), u)
    return np.ascontiguousarray(u)


def circuit_gates(circ) -> np.ndarray:
    return gates(circ.cliff, circ.tmask)


def _flat(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, np.complex128))
    return np.ascontiguousarray(u.view(np.float64).reshape(-1))


# --------------------------------------------------------------------------
# Amplitudes
# --------------------------------------------------------------------------

def _phases(n: int, d: int, phase):
    """None, or the (d, n-1) controlled-phase angles as a flat C array."""
    if phase is None:
        return None
    ph = np.ascontiguousarray(np.asarray(phase, np.float64).reshape(d, n - 1))
    return ph


def sv_state(n: int, d: int, u: np.ndarray, phase=None) -> np.ndarray:
    """Full state U|0^n> (2^n complex128, basis index bit q = x_q). phase:
    None (CZ entanglers) or (d, n-1) angles, phase[l, i] the controlled phase
    diag(1, 1, 1, e^(i phase)) on (i, i+1) in layer l (entries of uncoupled
    pairs are ignored)."""
    lib = _load()
    fu = _flat(u)
    assert fu.size == (d + 1) * n * 8
    ph = _phases(n, d, phase)
    out = np.empty(2 << n, np.float64)
    rc = lib.tbo_sv_state(n, d, _dptr(fu), None if ph is None else ph.ctypes.data, _dptr(out))
    if rc:
        raise RuntimeError(f"tbo_sv_state failed ({rc})")
    return out.view(np.complex128)


def basis_index(bits: np.ndarray) -> np.ndarray:
    bits = np.atleast_2d(np.asarray(bits, np.int64))
    return (bits << np.arange(bits.shape[1], dtype=np.int64)).sum(axis=1)


def sv_amplitudes(n: int, d: int, u: np.ndarray, bits: np.ndarray, phase=None) -> np.ndarray:
    return sv_state(n, d, u, phase)[basis_index(bits)]


def nb_amplitudes(n: int, d: int, u: np.ndarray, bits: np.ndarray,
                  return_peak: bool = False):
    """Naive boundary contraction, one bitstring at a time."""
    lib = _load()
    fu = _flat(u)
    assert fu.size == (d + 1) * n * 8
    bits = np.ascontiguousarray(np.atleast_2d(bits).astype(np.uint8))
    out = np.empty((bits.shape[0], 2), np.float64)
    peak = ctypes.c_int(0)
    peaks = []
    for i in range(bits.shape[0]):
        row = np.ascontiguousarray(bits[i])
        o = np.empty(2, np.float64)
        rc = lib.tbo_nb_amplitude(n, d, _dptr(fu), _u8ptr(row), _dptr(o), ctypes.byref(peak))
        if rc:
            raise RuntimeError(f"tbo_nb_amplitude failed ({rc})")
        out[i] = o
        peaks.append(peak.value)
    amps = out.view(np.complex128).reshape(-1)
    return (amps, max(peaks) if peaks else 0) if return_peak else amps


def feynman_amplitude(n: int, d: int, u: np.ndarray, x) -> complex:
    lib = _load()
    fu = _flat(u)
    xb = np.ascontiguousarray(np.asarray(x, np.uint8))
    o = np.empty(2, np.float64)
    rc = lib.tbo_feynman(n, d, _dptr(fu), _u8ptr(xb), _dptr(o))
    if rc:
        raise RuntimeError(f"tbo_feynman failed ({rc})")
    return complex(o[0], o[1])


def kron_state(n: int, d: int, u: np.ndarray, phase=None) -> np.ndarray:
    """U|0^n> from explicit 2^n x 2^n matrices: each slot is the Kronecker
    product of its one-qubit gates, each entangling layer the product of its
    two-qubit gates, each the 4x4 diag(1, 1, 1, w) (w = -1 for CZ, e^(i phase)
    otherwise) embedded by Kronecker products with identities. Basis index bit
    q = qubit q, so qubit n-1 is the leftmost Kronecker factor."""
    u = np.asarray(u, np.complex128)
    if phase is not None:
        phase = np.asarray(phase, np.float64).reshape(d, n - 1)
    dim = 1 << n
    idx = np.arange(dim)
    state = np.zeros(dim, np.complex128)
    state[0] = 1.0
    for t in range(d + 1):
        m = np.ones((1, 1), np.complex128)
        for q in reversed(range(n)):
            m = np.kron(m, u[t, q])
        state = m @ state
        if t < d:
            layer = np.eye(dim, dtype=np.complex128)
            for i0 in range(t % 2, n - 1, 2):
                w = -1.0 if phase is None else np.exp(1j * phase[t, i0])
                g = np.diag([1.0, 1.0, 1.0, w]).astype(np.complex128)  # basis (q_(i0+1), q_i0)
                full = np.kron(np.kron(np.eye(1 << (n - i0 - 2)), g), np.eye(1 << i0))
                layer = full @ layer
            state = layer @ state
    return state


def tableau_probability(circ, x) -> float:
    """|<x|U|0^n>|^2 of a Clifford-only circuit (T gates must be absent)."""
    if np.any(circ.tmask):
        raise ValueError("tableau needs a Clifford-only circuit (no T)")
    lib = _load()
    cl = np.ascontiguousarray(circ.cliff.astype(np.uint8))
    xb = np.ascontiguousarray(np.asarray(x, np.uint8))
    p = ctypes.c_double(0.0)
    rc = lib.tbo_tableau_prob(circ.n, circ.d, _u8ptr(cl), _u8ptr(xb), ctypes.byref(p))
    if rc:
        raise RuntimeError(f"tbo_tableau_prob failed ({rc})")
    return float(p.value)


def closed_form_hdiag(circ, bits: np.ndarray, phase=None) -> np.ndarray:
    """Exact amplitudes of an H / diagonal / H circuit.

    With H on every qubit at slot 0 and slot d and only diagonal gates in
    between (Cliffords I, Z, S, Z.S and T), everything between the two H layers
    commutes and multiplies |y> by exp(i theta.y) exp(i sum_e Phi_e y_i y_(i+1)),
    where theta_q collects the diagonal phases of qubit q and Phi_e the angles
    of the entangling gates on edge e (pi per CZ, so Phi_e = pi m_e with m_e the
    number of its CZ layers; phase[l, i] per gate otherwise). Hence
        psi(x) = 2^-n sum_y exp(i theta.y) exp(i sum_e Phi_e y_i y_(i+1)) (-1)^(x.y),
    evaluated with a 2x2 transfer matrix along the chain."""
    n, d = circ.n, circ.d
    tab = clifford_table()
    cl = circ.cliff.astype(np.int64)
    if not (np.all(cl[0] == 4) and np.all(cl[d] == 4)):
        raise ValueError("slots 0 and d must be H on every qubit")
    theta = np.zeros(n)
    for t in range(1, d):
        for q in range(n):
            c = tab[cl[t, q]]
            if abs(c[0, 1]) > 1e-12 or abs(c[1, 0]) > 1e-12 or abs(c[0, 0] - 1) > 1e-12:
                raise ValueError("interior slots must be diagonal with (0,0) entry 1")
            theta[q] += np.angle(c[1, 1])
    theta += (np.pi / 4) * circ.tmask.sum(axis=0)
    if phase is None:
        m = np.array([sum(1 for l in range(d) if l % 2 == i % 2) % 2 for i in range(n - 1)])
        w_edge = np.where(m == 1, -1.0, 1.0).astype(np.complex128)
    else:
        phase = np.asarray(phase, np.float64).reshape(d, n - 1)
        big_phi = np.array([sum(phase[l, i] for l in range(d) if l % 2 == i % 2) for i in range(n - 1)])
        w_edge = np.exp(1j * big_phi)
    bits = np.atleast_2d(bits)
    out = np.empty(bits.shape[0], np.complex128)
    for b, x in enumerate(bits):
        ph = np.exp(1j * theta) * np.where(x == 1, -1.0, 1.0)
        v = np.array([1.0 + 0j, ph[0]])
        for q in range(1, n):
            v = np.array([v[0] + v[1], (v[0] + w_edge[q - 1] * v[1]) * ph[q]])
        out[b] = (v[0] + v[1]) / (2.0 ** n)
    return out


EULER_GAMMA = 0.57721566490153286060651209


def log_xeb(amps: np.ndarray, n: int) -> float:
    """F = gamma + n ln 2 + (1/N) sum_i ln p(x_i), p = |psi|^2 (Sec. 5.2, normalized log-XEB equation)."""
    p = np.abs(np.asarray(amps, np.complex128)) ** 2
    return float(EULER_GAMMA + n * np.log(2.0) + np.mean(np.log(p)))


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    """||a - ref||_2 / ||ref||_2 over a batch."""
    a = np.asarray(a, np.complex128)
    ref = np.asarray(ref, np.complex128)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB_PATH)


def alg1_cost(n: int, d: int) -> tuple:
    """(W, log2 C) of the constructive path of Algorithm 1 (Sec. 3.1) for the
    amplitude network of an n-qubit, depth-d brickwork circuit (Sec. 2.2).

    The network (Sec. 2.2): every CZ is split into two rank-3 halves, one per
    qubit, joined by a bond of dimension chi = 2; the halves of one qubit are
    chained in time by legs of dimension 2; the input state, the output
    projector and the one-qubit gates are absorbed, so the first and last
    half of a qubit carry one time leg. Every leg has dimension 2, so a
    tensor's log2 size is its number of legs.

    The path: the halves in FixedSweepOrder -- qubit rows 0..n-1, row 0 and
    odd rows in forward time, even rows >= 2 in reversed time (the paper's
    "reverse time on even-numbered rows" under the layer convention that
    layer l couples (i, i+1) for i = l mod 2). The boundary B starts as the
    first tensor; the next tensor X is contracted into B if the result has at
    most h = ceil(d/2) legs, otherwise X is first contracted with the tensor
    after it and the pair is contracted into B. A pairwise contraction of
    A_IK B_KJ costs |I||J||K| = 2^(#legs of A union B) (Sec. 2.2); W is the
    largest log2 size of any tensor the path creates."""
    h = (d + 1) // 2
    rows = []
    for q in range(n):
        layers = [l for l in range(d)
                  if (l % 2 == q % 2 and q + 1 < n) or (q >= 1 and l % 2 == (q - 1) % 2)]
        legs = []
        for i, l in enumerate(layers):
            lo = q if l % 2 == q % 2 else q - 1          # the bond's upper qubit is lo + 1
            t = {("bond", l, lo)}
            if i > 0:
                t.add(("time", q, i - 1))
            if i + 1 < len(layers):
                t.add(("time", q, i))
            legs.append(frozenset(t))
        if q >= 2 and q % 2 == 0:
            legs.reverse()
        rows.append(legs)
    order = [t for r in rows for t in r]
    if not order:
        return 0, float("-inf")
    costs = []
    width = 0
    B = set(order[0])
    width = max(width, len(B))
    i = 1
    while i < len(order):
        X = order[i]
        if len(B ^ X) <= h:
            costs.append(len(B | X))
            B = B ^ X
            i += 1
        else:
            Y = order[i + 1]
            costs.append(len(X | Y))
            Cxy = X ^ Y
            width = max(width, len(Cxy))
            costs.append(len(B | Cxy))
            B = B ^ Cxy
            i += 2
        width = max(width, len(B))
    m = max(costs)
    log2c = m + float(np.log2(sum(2.0 ** (c - m) for c in costs)))
    return width, log2c
