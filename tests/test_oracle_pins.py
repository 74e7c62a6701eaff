"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics,
never against the oracle itself.

Each check is chosen so that a plausible mistake fails it:
  * a wrong CZ parity or sign            -> hand-computed 3-qubit states, Kronecker product
  * a transposed gate or wrong gate order -> Kronecker product, brute force
  * a dropped or doubled term in the row contraction -> brute force, norm = 1
  * a wrong Clifford decomposition in the tableau -> tableau vs Kronecker product
  * a wrong T phase or T/Clifford order   -> explicit matrix checks, closed form
  * a controlled phase on the wrong pair or layer, or a conjugated one
                                          -> worked example, Kronecker product with
                                             random angles, phi = pi (CZ) and phi = 0
                                             (product state), closed form
"""
import itertools

import numpy as np
import pytest

import workloads as W


def _all_bits(n):
    return np.array([[(i >> q) & 1 for q in range(n)] for i in range(1 << n)], np.uint8)


# ---------------------------------------------------------------- gate table

def test_clifford_table_named_entries(oracle_mod):
    tab = oracle_mod.clifford_table()
    s = np.sqrt(0.5)
    np.testing.assert_allclose(tab[0], np.eye(2))
    np.testing.assert_allclose(tab[1], [[0, 1], [1, 0]])
    np.testing.assert_allclose(tab[2], [[0, -1j], [1j, 0]])
    np.testing.assert_allclose(tab[3], [[1, 0], [0, -1]])
    np.testing.assert_allclose(tab[4], [[s, s], [s, -s]])
    np.testing.assert_allclose(tab[8], [[1, 0], [0, 1j]])
    np.testing.assert_allclose(tab[11], [[1, 0], [0, -1j]])  # Z.S = S^dagger


def test_clifford_table_is_the_clifford_group(oracle_mod):
    tab = oracle_mod.clifford_table()
    paulis = [np.array(p, np.complex128) for p in
              ([[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]])]
    reps = []
    for c in tab:
        np.testing.assert_allclose(c.conj().T @ c, np.eye(2), atol=1e-14)
        for p in paulis[0], paulis[2]:
            img = c @ p @ c.conj().T
            assert any(np.allclose(img, sg * q) for q in paulis for sg in (1, -1)), \
                "Clifford must map X and Z to signed Paulis"
        # representative modulo global phase
        k = np.argmax(np.abs(c.reshape(-1)) > 1e-9)
        reps.append(c / (c.reshape(-1)[k] / abs(c.reshape(-1)[k])))
    for a, b in itertools.combinations(range(24), 2):
        assert not np.allclose(reps[a], reps[b], atol=1e-9), (a, b)


def test_t_gate_and_slot_order(oracle_mod):
    t = oracle_mod.T_GATE
    np.testing.assert_allclose(t, np.diag([1, np.exp(1j * np.pi / 4)]))
    np.testing.assert_allclose(np.linalg.matrix_power(t, 8), np.eye(2), atol=1e-14)
    cliff = np.array([[4, 2], [5, 9]], np.uint8)          # d = 1, n = 2
    tmask = np.array([[1, 0]], np.uint8)
    u = oracle_mod.gates(cliff, tmask)
    tab = oracle_mod.clifford_table()
    np.testing.assert_allclose(u[0, 0], t @ tab[4])        # T after the Clifford
    np.testing.assert_allclose(u[0, 1], tab[2])
    np.testing.assert_allclose(u[1, 0], tab[5])            # slot d never gets T


# ------------------------------------------------------------ state vector

def test_brickwork_parity_hand_computed(oracle_mod):
    """n=3, d=2, H on every qubit at slot 0, identity elsewhere. Layer 0
    couples (0,1) only, layer 1 couples (1,2) only, so the state is
    2^-3/2 sum_y (-1)^(y0 y1 + y1 y2) |y>."""
    n, d = 3, 2
    cliff = np.zeros((d + 1, n), np.uint8)
    cliff[0, :] = 4
    u = oracle_mod.gates(cliff, np.zeros((d, n), np.uint8))
    psi = oracle_mod.sv_state(n, d, u)
    exp = np.array([(-1) ** (((y >> 0) & 1) * ((y >> 1) & 1) + ((y >> 1) & 1) * ((y >> 2) & 1))
                    for y in range(8)]) / np.sqrt(8)
    np.testing.assert_allclose(psi, exp, atol=1e-15)
    # d = 1: only (0,1) is coupled
    u1 = oracle_mod.gates(cliff[:2], np.zeros((1, n), np.uint8))
    psi1 = oracle_mod.sv_state(n, 1, u1)
    exp1 = np.array([(-1) ** (((y >> 0) & 1) * ((y >> 1) & 1)) for y in range(8)]) / np.sqrt(8)
    np.testing.assert_allclose(psi1, exp1, atol=1e-15)


@pytest.mark.parametrize("n,d", [(1, 0), (1, 3), (2, 1), (3, 4), (4, 5), (5, 6), (6, 3)])
def test_sv_matches_kronecker_product(oracle_mod, n, d):
    u = W.random_unitaries(n, d, 100 + 10 * n + d)
    np.testing.assert_allclose(oracle_mod.sv_state(n, d, u), oracle_mod.kron_state(n, d, u),
                               atol=1e-13)


@pytest.mark.parametrize("n,d", [(2, 3), (3, 4), (4, 4), (3, 5), (5, 3), (4, 1)])
def test_sv_matches_brute_force_path_sum(oracle_mod, n, d):
    u = W.random_unitaries(n, d, 200 + 10 * n + d)
    psi = oracle_mod.sv_state(n, d, u)
    rng = np.random.default_rng(n * 31 + d)
    for _ in range(3):
        x = rng.integers(0, 2, n).astype(np.uint8)
        f = oracle_mod.feynman_amplitude(n, d, u, x)
        assert abs(f - psi[oracle_mod.basis_index(x)[0]]) < 1e-13


# ------------------------------------------------------- naive boundary sweep

@pytest.mark.parametrize("n,d", [(1, 4), (2, 2), (3, 3), (4, 7), (5, 8), (6, 6), (7, 9),
                                 (8, 10), (9, 11), (4, 0), (5, 1)])
def test_nb_matches_state_vector(oracle_mod, n, d):
    u = W.random_unitaries(n, d, 300 + 10 * n + d)
    bits = _all_bits(n) if n <= 6 else np.random.default_rng(n).integers(0, 2, (40, n)).astype(np.uint8)
    np.testing.assert_allclose(oracle_mod.nb_amplitudes(n, d, u, bits),
                               oracle_mod.sv_amplitudes(n, d, u, bits), atol=1e-13)


@pytest.mark.parametrize("n,d", [(4, 8), (6, 7), (8, 6), (7, 12)])
def test_nb_probabilities_sum_to_one(oracle_mod, n, d):
    u = W.random_unitaries(n, d, 400 + n + d)
    amps = oracle_mod.nb_amplitudes(n, d, u, _all_bits(n))
    assert abs(np.sum(np.abs(amps) ** 2) - 1.0) < 1e-12


def test_nb_brute_force_directly(oracle_mod):
    n, d = 3, 6
    u = W.random_unitaries(n, d, 77)
    for x in _all_bits(n)[::3]:
        assert abs(oracle_mod.nb_amplitudes(n, d, u, x[None])[0]
                   - oracle_mod.feynman_amplitude(n, d, u, x)) < 1e-13


def test_nb_width_is_temporal(oracle_mod):
    """The row-by-row contraction never holds more than ceil(d/2) stored layer
    values plus the wire and one freshly copied value (the temporal width of
    Sec. 2.2 is ceil(d/2))."""
    for n, d in [(6, 8), (7, 9), (8, 12)]:
        u = W.random_unitaries(n, d, 5)
        _, peak = oracle_mod.nb_amplitudes(n, d, u, np.zeros((1, n), np.uint8), return_peak=True)
        h = (d + 1) // 2
        assert h <= peak <= h + 2


# -------------------------------------------------------------- tableau

@pytest.mark.parametrize("n,d,seed", [(5, 6, 1), (8, 7, 2), (10, 9, 3), (6, 12, 4)])
def test_tableau_matches_state_vector(oracle_mod, n, d, seed):
    c = W.random_circuit(n, d, 0, 0, seed)
    psi = oracle_mod.sv_state(n, d, oracle_mod.circuit_gates(c))
    bits = _all_bits(n)
    p = np.array([oracle_mod.tableau_probability(c, x) for x in bits])
    np.testing.assert_allclose(p, np.abs(psi) ** 2, atol=1e-13)
    nz = p[p > 0]
    r = -np.log2(nz)
    assert np.allclose(r, np.round(r)) and np.allclose(nz, nz[0]), "stabilizer |amp|^2 in {0, 2^-r}"
    assert abs(p.sum() - 1.0) < 1e-12


def test_tableau_rejects_t(oracle_mod):
    c = W.random_circuit(4, 4, 2, 1, 9)
    with pytest.raises(ValueError):
        oracle_mod.tableau_probability(c, c.bits[0])


# ---------------------------------------------------------- closed form

@pytest.mark.parametrize("n,d", [(6, 4), (7, 6), (8, 8), (9, 10), (5, 7), (10, 3)])
def test_closed_form_matches_state_vector(oracle_mod, n, d):
    c = W.hdiag_circuit(n, d, max(1, n * d // 10), 0, 50 + n + d)
    bits = _all_bits(n)
    np.testing.assert_allclose(oracle_mod.closed_form_hdiag(c, bits),
                               oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), bits),
                               atol=1e-14)


def test_closed_form_product_when_d_is_0_mod_4(oracle_mod):
    """For d = 0 (mod 4) every edge sees an even number of CZ layers, so the
    amplitude factorises: psi(x) = prod_q (1 + e^(i theta_q) (-1)^(x_q)) / 2."""
    c = W.hdiag_circuit(70, 64, 426, 8, 7)
    tab = oracle_mod.clifford_table()
    theta = np.zeros(70)
    for t in range(1, 64):
        theta += np.angle(tab[c.cliff[t].astype(int), 1, 1])
    theta += np.pi / 4 * c.tmask.sum(axis=0)
    # keep every factor away from zero so that the comparison is relative:
    # x_q picks the larger of |1 + e^(i theta_q)| and |1 - e^(i theta_q)|
    rng = np.random.default_rng(3)
    big = (np.cos(theta) < 0).astype(np.uint8)
    bits = np.array([big if k == 0 else np.where(rng.random(70) < 0.2, 1 - big, big)
                     for k in range(8)], np.uint8)
    bits = np.where(np.abs(np.cos(theta / 2)) > 1e-6, bits, 1)       # never a zero factor
    bits = np.where(np.abs(np.sin(theta / 2)) > 1e-6, bits, 0).astype(np.uint8)
    exp = np.prod((1 + np.exp(1j * theta) * np.where(bits == 1, -1, 1)) / 2, axis=1)
    assert np.all(np.abs(exp) > 1e-40)
    np.testing.assert_allclose(oracle_mod.closed_form_hdiag(c, bits), exp, rtol=1e-12, atol=0)


@pytest.mark.parametrize("d", [63, 65])
def test_closed_form_pair_product_for_odd_d(oracle_mod, d):
    """For odd d, edge (i, i+1) sees ceil(d/2) CZ layers when i is even and
    floor(d/2) when i is odd, so exactly one parity of edges keeps a CZ and the
    amplitude at n = 70 is a product of disjoint pair factors (and single-qubit
    factors at the chain ends), each a four-term sum written out here:
    f(x_a, x_b) = 1/4 sum_(y,y') e^(i(th_a y + th_b y')) (-1)^(y y' + x_a y + x_b y')."""
    n = 70
    c = W.hdiag_circuit(n, d, int(round(0.095 * n * d)), 6, 8 + d)
    tab = oracle_mod.clifford_table()
    theta = np.zeros(n)
    for t in range(1, d):
        theta += np.angle(tab[c.cliff[t].astype(int), 1, 1])
    theta += np.pi / 4 * c.tmask.sum(axis=0)
    kept = 0 if ((d + 1) // 2) % 2 == 1 else 1  # parity of the edges with an odd CZ count
    assert ((d + 1) // 2 if kept == 0 else d // 2) % 2 == 1

    def single(th, x):
        return (1 + np.exp(1j * th) * (-1) ** x) / 2

    def pair(ta, tb, xa, xb):
        tot = 0
        for y in (0, 1):
            for yp in (0, 1):
                tot += np.exp(1j * (ta * y + tb * yp)) * (-1) ** (y * yp + xa * y + xb * yp)
        return tot / 4

    groups = ([(0,)] if kept == 1 else []) + [(q, q + 1) for q in range(kept, n - 1, 2)]
    if groups[-1][-1] < n - 1:
        groups.append((n - 1,))

    def factor(g, x):
        return single(theta[g[0]], x[g[0]]) if len(g) == 1 else pair(theta[g[0]], theta[g[1]], x[g[0]], x[g[1]])

    # bitstrings whose factors are all far from zero, so that the comparison is
    # relative: each group takes its largest factor, or on a random fifth of
    # the groups its second largest
    rng = np.random.default_rng(d)
    bits = np.zeros((6, n), np.int64)
    for b in range(6):
        for g in groups:
            opts = []
            for v in range(1 << len(g)):
                x = bits[b].copy()
                for j, q in enumerate(g):
                    x[q] = (v >> j) & 1
                opts.append((abs(factor(g, x)), v))
            opts.sort(reverse=True)
            v = opts[1][1] if (b > 0 and rng.random() < 0.2) else opts[0][1]
            for j, q in enumerate(g):
                bits[b, q] = (v >> j) & 1
    exp = np.array([np.prod([factor(g, x) for g in groups]) for x in bits])
    got = oracle_mod.closed_form_hdiag(c, bits.astype(np.uint8))
    np.testing.assert_allclose(got, exp, rtol=1e-10, atol=0)


def test_identity_circuit(oracle_mod):
    for n, d in [(5, 6), (8, 9)]:
        c = W.identity_circuit(n, d, 10, 3)
        u = oracle_mod.circuit_gates(c)
        exp = np.array([1.0 if not x.any() else 0.0 for x in c.bits])
        np.testing.assert_allclose(oracle_mod.nb_amplitudes(n, d, u, c.bits), exp, atol=1e-15)


# ------------------------------------------------ controlled-phase entanglers

def test_controlled_phase_worked_example(oracle_mod):
    """H on both qubits, then diag(1, 1, 1, e^(i phi)): the state is
    (|00> + |01> + |10> + e^(i phi)|11>) / 2."""
    phi = 0.7
    u = np.tile(np.eye(2, dtype=np.complex128), (2, 2, 1, 1))
    u[0, :] = np.array([[1, 1], [1, -1]]) / np.sqrt(2.0)
    exp = np.array([1, 1, 1, np.exp(1j * phi)]) / 2.0
    ph = np.array([[phi]])
    np.testing.assert_allclose(oracle_mod.sv_state(2, 1, u, ph), exp, atol=1e-15)
    np.testing.assert_allclose(oracle_mod.kron_state(2, 1, u, ph), exp, atol=1e-15)


@pytest.mark.parametrize("n,d", [(2, 3), (3, 4), (4, 5), (5, 6), (6, 3), (7, 4)])
def test_controlled_phase_sv_matches_kronecker_product(oracle_mod, n, d):
    u = W.random_unitaries(n, d, 300 + n + d)
    ph = W.random_phases(n, d, 400 + n + d)
    np.testing.assert_allclose(oracle_mod.sv_state(n, d, u, ph), oracle_mod.kron_state(n, d, u, ph),
                               atol=1e-13)


def test_controlled_phase_pi_is_cz_and_zero_is_a_product(oracle_mod):
    n, d = 6, 7
    u = W.random_unitaries(n, d, 77)
    np.testing.assert_allclose(oracle_mod.sv_state(n, d, u, np.full((d, n - 1), np.pi)),
                               oracle_mod.sv_state(n, d, u), atol=1e-14)
    # no entanglement: the state is the Kronecker product of each qubit's chain
    psi = oracle_mod.sv_state(n, d, u, np.zeros((d, n - 1)))
    cols = []
    for q in range(n):
        v = np.array([1.0, 0.0], np.complex128)
        for t in range(d + 1):
            v = u[t, q] @ v
        cols.append(v)
    prod = np.ones(1, np.complex128)
    for q in reversed(range(n)):
        prod = np.kron(prod, cols[q])
    np.testing.assert_allclose(psi, prod, atol=1e-14)


@pytest.mark.parametrize("n,d", [(6, 4), (7, 7), (8, 9), (9, 6)])
def test_controlled_phase_closed_form_matches_state_vector(oracle_mod, n, d):
    c = W.hdiag_circuit(n, d, 3 * n, 0, 60 + n + d)
    ph = W.random_phases(n, d, 70 + n + d)
    bits = _all_bits(n)
    ref = oracle_mod.sv_amplitudes(n, d, oracle_mod.circuit_gates(c), bits, ph)
    np.testing.assert_allclose(oracle_mod.closed_form_hdiag(c, bits, ph), ref, atol=1e-13)


def test_zz_rotation_is_a_controlled_phase_up_to_one_qubit_gates(oracle_mod):
    """exp(i c ZZ) = e^(-ic) (Rz(-2c) x Rz(-2c)) diag(1, 1, 1, e^(4ic)): a
    brickwork of ZZ rotations equals the controlled-phase brickwork with the
    Rz folded into the next slot (the statement that covers every entangler of
    operator Schmidt rank 2 up to one-qubit gates)."""
    n, d = 4, 3
    u = W.random_unitaries(n, d, 91)
    c = W.random_phases(n, d, 92) - np.pi
    rz = lambda t: np.diag([np.exp(-0.5j * t), np.exp(0.5j * t)])
    # reference: explicit 2^n matrices with exp(i c ZZ) entanglers
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
            for i0 in range(t % 2, n - 1, 2):
                zz = (1 - 2 * ((idx >> i0) & 1)) * (1 - 2 * ((idx >> (i0 + 1)) & 1))
                state = np.exp(1j * c[t, i0] * zz) * state
    # controlled phases 4c, Rz(-2c) folded into slot t+1 of both qubits, global phases
    u2 = u.copy()
    glob = 1.0 + 0j
    for t in range(d):
        for i0 in range(t % 2, n - 1, 2):
            u2[t + 1, i0] = u2[t + 1, i0] @ rz(-2 * c[t, i0])
            u2[t + 1, i0 + 1] = u2[t + 1, i0 + 1] @ rz(-2 * c[t, i0])
            glob *= np.exp(-1j * c[t, i0])
    got = glob * oracle_mod.sv_state(n, d, u2, 4 * c)
    np.testing.assert_allclose(got, state, atol=1e-13)


# ---------------------------------------------------------------- log-XEB

def test_log_xeb_definition(oracle_mod):
    n = 20
    # uniform distribution: every ln p = -n ln 2, so F = gamma
    amps = np.full(100, 2.0 ** (-n / 2), np.complex128)
    assert abs(oracle_mod.log_xeb(amps, n) - oracle_mod.EULER_GAMMA) < 1e-12
    # Porter-Thomas draws p = z / 2^n, z ~ Exp(1): E[ln z] = -gamma, so F ~ 0
    rng = np.random.default_rng(11)
    N = 200000
    z = rng.exponential(1.0, N)
    amps = np.sqrt(z / 2.0 ** n).astype(np.complex128)
    sd = np.pi / np.sqrt(6.0) / np.sqrt(N)
    assert abs(oracle_mod.log_xeb(amps, n)) < 5 * sd


# ------------------------------------------------- Algorithm 1 cost counter

def _paper_numbers():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_alg1_cost_matches_the_paper_at_n70_d70(oracle_mod):
    """Sec. 6.2 / 6.3 print (W, log2 C) = (35, 48.22) for the chi=2 open chain
    at n = d = 70. A wrong sweep direction, a dropped bond or time leg, or a
    cost other than |I||J||K| moves one of the two numbers."""
    g = _paper_numbers()["width_cost_open_chi2_n70_d70"]
    w, c = oracle_mod.alg1_cost(g["n"], g["d"])
    assert w == g["W"]
    assert abs(c - g["log2_C"]) < g["log2_C_tolerance"]


def test_alg1_width_is_proposition_1(oracle_mod):
    """Proposition 1: the constructive path has width ceil(d/2) for n >= 4 and
    7 <= d <= 2n (the values listed in the paper for n = 70, and a spread of
    smaller even and odd cases)."""
    g = _paper_numbers()["constructive_width"]
    for d in g["d"]:
        assert oracle_mod.alg1_cost(g["n"], d)[0] == (d + 1) // 2, d
    for n, d in [(4, 7), (5, 9), (8, 16), (12, 9), (20, 33), (30, 40), (33, 66)]:
        assert oracle_mod.alg1_cost(n, d)[0] == (d + 1) // 2, (n, d)


def test_alg1_cost_brute_force_on_a_tiny_network(oracle_mod):
    """n = 2, d = 2: two qubits, one CZ in layer 0 only (layer 1 couples (1, 2),
    which does not exist). Each qubit has one half with only the bond leg:
    B = {bond} (1 leg), X = {bond}: one contraction of two 1-leg tensors over
    the shared bond, |I||J||K| = 1 * 1 * 2 = 2, so log2 C = 1 and W = 1."""
    w, c = oracle_mod.alg1_cost(2, 2)
    assert w == 1 and abs(c - 1.0) < 1e-12
