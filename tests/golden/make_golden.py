"""Writes the stored QAOA amplitudes under tests/golden/ from the CPU oracle.

Each fixture is one seeded random 3-regular QAOA instance (the workload of
Sec. IV: random 3-regular graphs, depth p) with its edges, angles and a set of
seeded bit strings, and the amplitudes a(x) = <x| U_B(beta_p) U_C(gamma_p) ...
U_B(beta_1) U_C(gamma_1) H^n |0^n> (Sec. II, the circuit the tensor network of
Sec. II.A encodes) from the oracle's state vector.  The state vector is itself
pinned by the closed forms and library cross-checks of tests/test_oracle.py;
the files freeze its values so that later changes of the oracle or of the
instance generator show up, and give the device path fixed inputs.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2010_14962_gb300 import instances as I  # noqa: E402

FIXTURES = [
    # (file, n, p, instance seed, bit strings, bit-string seed)
    ("qaoa16_p1_seed1.txt", 16, 1, 1, 32, 11),
    ("qaoa14_p2_seed4.txt", 14, 2, 4, 32, 12),
    ("qaoa12_p3_seed7.txt", 12, 3, 7, 32, 13),
]


def write(name, n, p, seed, nx, xseed):
    inst = I.qaoa_instance(n, p, seed)
    sv = O.statevector(n, inst.edges, inst.gamma, inst.beta)
    xs = I.bitstrings(n, nx, xseed)
    lines = [
        "# QAOA amplitudes a(x) of a seeded random 3-regular instance (Sec. II / Sec. IV workload),",
        "# from the CPU oracle's state vector (tests/golden/make_golden.py). x[i] = bit of qubit i.",
        f"n {n}",
        f"p {p}",
        "gamma " + " ".join(repr(float(g)) for g in inst.gamma),
        "beta " + " ".join(repr(float(b)) for b in inst.beta),
        "edges " + " ".join(f"{a}-{b}" for a, b in np.asarray(inst.edges)),
        f"norm {float(np.sum(np.abs(sv) ** 2))!r}",
    ]
    for x in xs:
        a = sv[O.bits_to_int(x)]
        lines.append("x " + "".join(str(int(v)) for v in x) + f" {float(a.real)!r} {float(a.imag)!r}")
    with open(os.path.join(HERE, name), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    for fx in FIXTURES:
        write(*fx)
        print("wrote", fx[0])
