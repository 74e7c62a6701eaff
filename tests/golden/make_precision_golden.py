"""Write tests/golden/precision_n32_d48.json: FP64 amplitudes of the
width-24 precision case (n = 32, d = 48, 146 T gates, random Cliffords, the
seeded generator's slice of the n = 70, d = 64 shape) computed by the oracle's
naive boundary contraction. The circuit itself is stored with the values so
that readers need no random generator.

Context: the paper measures the precision of complex64 against complex128
(Sec. 5.1); these values are the complex128-side reference for the GPU's
FP32 and split-precision tensor-core paths.

    python tests/golden/make_precision_golden.py [n_bitstrings]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main(nb: int = 12) -> None:
    oracle.build()
    c = W.slice_32_48(nb=nb)
    u = oracle.circuit_gates(c)
    t0 = time.time()
    amps = oracle.nb_amplitudes(c.n, c.d, u, c.bits)
    out = {
        "what": "FP64 naive-boundary amplitudes <x|U|0^n> of an open 1D brickwork CZ circuit "
                "(Sec. 2.1 circuit family; Sec. 5.1 complex128 reference)",
        "generator": "workloads.slice_32_48(nb=%d), oracle.nb_amplitudes" % nb,
        "n": c.n, "d": c.d, "n_t": c.n_t,
        "cliff": c.cliff.tolist(), "tmask": c.tmask.tolist(), "bits": c.bits.tolist(),
        "amps": [[float(a.real), float(a.imag)] for a in amps],
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": oracle.num_threads(),
    }
    with open(os.path.join(HERE, "precision_n32_d48.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 12)
