"""Write tests/golden/closed_form_n70_d64.json: exact amplitudes of the
n = 70, d = 64 H / diagonal / H circuit with 426 T gates (the seeded
generator's hdiag_circuit(70, 64, 426, 0, 4100)), from the oracle's closed
form. Between the two H layers every gate is diagonal, so the amplitude is a
product of per-qubit factors (d = 0 mod 4: every edge carries an even number
of CZ layers). The bitstrings are chosen so that no factor is small (each
qubit's bit takes the value that makes |1 + e^(i theta_q) (-1)^(x_q)| the
larger, flipped with probability 1/4; a qubit with a vanishing factor takes
the value that keeps it).

    python tests/golden/make_closed_form_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main(nb: int = 4) -> None:
    c = W.hdiag_circuit(70, 64, 426, 0, 4100)
    tab = oracle.clifford_table()
    theta = np.zeros(c.n)
    for t in range(1, c.d):
        theta += np.angle(tab[c.cliff[t].astype(int), 1, 1])
    theta += np.pi / 4 * c.tmask.sum(axis=0)
    big = (np.cos(theta) < 0).astype(np.uint8)
    rng = np.random.default_rng(7)
    bits = np.array([np.where(rng.random(c.n) < 0.25, 1 - big, big) for _ in range(nb)], np.uint8)
    # a qubit whose factor (1 + e^(i theta) (-1)^x) / 2 vanishes for one value
    # of x takes the other value
    bits = np.where(np.abs(np.cos(theta / 2)) > 1e-6, bits, 1)
    bits = np.where(np.abs(np.sin(theta / 2)) > 1e-6, bits, 0).astype(np.uint8)
    amps = oracle.closed_form_hdiag(c, bits)
    out = {
        "what": "exact amplitudes of an H / diagonal / H brickwork circuit, n=70, d=64, 426 T "
                "(closed form; Sec. 2.1 circuit family)",
        "generator": "workloads.hdiag_circuit(70, 64, 426, 0, 4100), oracle.closed_form_hdiag",
        "n": c.n, "d": c.d, "n_t": c.n_t,
        "cliff": c.cliff.tolist(), "tmask": c.tmask.tolist(), "bits": bits.tolist(),
        "amps": [[float(a.real), float(a.imag)] for a in amps],
    }
    with open(os.path.join(HERE, "closed_form_n70_d64.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main()
